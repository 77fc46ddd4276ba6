// k_sda_dwt.cu -- SDA group sums (Sec. III-B) fused with the first level of
// the wavelet decomposition the denoiser starts with (Sec. II-A), for uint8
// frames whose padded width equals W (W * C a multiple of 16 bytes, 16-byte
// aligned rows and frames) and groups of at most 257 frames.
//
// A block owns 32*QG output columns of one group -- input columns
// 2*cq0 .. 2*cq0 + 64*QG - 1 of all C channels plus the 6-column right halo
// of the 8-tap filters -- and walks down a strip of output rows, two input
// rows (one output row) per stage.  The frames of a stage arrive in slices of
// up to FB frames: every thread copies its share of the slice's 16-byte
// chunks (both rows, every frame of the slice) into shared memory with
// cp.async, and the copies of slice k+1 are issued as soon as slice k has
// landed, so they stay in flight through the summing of slice k and, at the
// end of a stage, through its hand-off and analysis.  Per stage:
//   1. thread (unit, sub) sums one chunk of one of the two rows over frames
//      sub, sub + NSUB, ... of each slice in packed 16-bit lanes (even and odd
//      bytes of each word, as the SDA kernel does) and leaves the packed
//      partial in shared memory;
//   2. barrier; the partials are added (exact: a lane holds at most
//      257 * 255 < 2^16) and de-interleaved into one float row per channel
//      over the block's span;
//   3. barrier; warp (c, g) -- channel c, output columns cq0 + 32g .. +31 --
//      writes its 64 columns of both rows to the SDA plane X (the MLE step
//      reads it), forms the row pass of both rows into its 8-row register
//      ring and, once the ring holds rows 2p..2p+7, the column pass and the
//      four level-1 subbands of output row p.
// Step 3 is the streaming analysis's arithmetic (dwt_rows.cuh) in the same
// order on the same exact integer sums, so the fused and the separate kernels
// give the same bits.
#include <algorithm>

#include "dwt_rows.cuh"

namespace prnu {
namespace {

constexpr int kMaxSlice = 56;  // frames per slice: two slice buffers of 3-channel blocks take 93 KB

template <int C, int QG>
struct FusedGeo {
    static constexpr int OWN = 64 * QG * C;          // owned bytes of a row
    static constexpr int OWNCH = OWN / 16;           // owned 16-byte chunks
    static constexpr int HALOCH = (6 * C + 15) / 16;  // chunks holding the 6-column halo
    static constexpr int NCH = OWNCH + HALOCH;       // chunks of a row
    static constexpr int NU = 2 * NCH;               // (row, chunk) units of a stage
    static constexpr int NW = C * QG;                // warps: (channel, 32 output columns)
    static constexpr int NT = 32 * NW;
    static constexpr int NSUB = NT / NU;             // frame subsets per unit
    static constexpr int SPAN = ((NCH * 16 + C - 1) / C + 1) & ~1;  // floats of one channel row
    static_assert(NSUB >= 1, "one thread per unit at least");
};

// even bytes (0, 2) and odd bytes (1, 3) of two words into the 16-bit lanes
// of ev / od: one byte permute per word and lane set, one three-input add
__device__ __forceinline__ void lanes_add2(uint32_t v, uint32_t w, uint32_t &ev, uint32_t &od) {
    ev = ev + __byte_perm(v, 0u, 0x4240) + __byte_perm(w, 0u, 0x4240);
    od = od + __byte_perm(v, 0u, 0x4341) + __byte_perm(w, 0u, 0x4341);
}

__device__ __forceinline__ void cp16(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// fb: frames per slice (<= kMaxSlice); dynamic shared memory holds two slices
// of NU x fb chunks
template <int C, int QG, class T>
__global__ void __launch_bounds__(FusedGeo<C, QG>::NT, 2) k_sda_dwt(SdaArgs s, AnaArgs a, int spr, int fb) {
    using FG = FusedGeo<C, QG>;
    extern __shared__ __align__(16) uint4 stg[];  // [2][fb][NU] chunks
    __shared__ __align__(16) uint32_t part[FG::NSUB][FG::NU][8];
    __shared__ __align__(16) float xs[C][2][FG::SPAN];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gi = blockIdx.y;  // group of the pass
    const int R2 = a.R >> 1, C2 = a.Cc >> 1;
    const int cq0 = blockIdx.x * 32 * QG;
    const int p0 = blockIdx.z * spr, pend = min(p0 + spr, R2);
    const int npr = pend - p0;
    const int rowbytes = s.W * C;
    // the group's frames: consecutive groups of d frames of one sequence, or
    // (multi-camera pass) the group's own descriptor
    const uint8_t *frames = s.frames;
    long long fstride = s.frame_stride, rpitch = s.row_pitch;
    int j0, j1, jmax;
    if (s.gd) {
        const GroupDesc &gdesc = s.gd[gi];
        frames = gdesc.frames;
        fstride = gdesc.frame_stride;
        rpitch = gdesc.row_pitch;
        j0 = 0;
        j1 = jmax = gdesc.n;
    } else {
        j0 = (s.g0 + gi) * s.d;
        j1 = min(s.m, j0 + s.d);
        jmax = s.m;
    }
    // owned bytes of this block (a multiple of 16) and the source of its halo:
    // the next bytes of the row, or the row start past the last column
    const int seg0 = 2 * cq0 * C;
    const int own = min(FG::OWN, rowbytes - seg0);
    const int ownch = own / 16;
    const bool halo_next = seg0 + own < rowbytes;
    // byte offset in the row of chunk k of the span (-1: past the halo)
    auto chunk_off = [&](int k) {
        if (k < ownch) return seg0 + 16 * k;
        if (k < ownch + FG::HALOCH) return halo_next ? seg0 + own + 16 * (k - ownch) : 16 * (k - ownch);
        return -1;
    };
    // source row of strip-relative input row t (periodic in the padded
    // height, mirrored into the frame)
    auto src_row = [&](int t) {
        int sy = mirror(wrap_near(2 * p0 + t, a.R), s.H);
        if (!PRNU_DCHECK(sy >= 0 && sy < s.H, sy)) sy = 0;
        return sy;
    };

    // the unit this thread copies and sums: chunk uch of row urow, frames
    // sub, sub + NSUB, ... of every slice (its own shared-memory slots, so a
    // slice needs no barrier: the thread waits for its own copies only)
    const int unit = tid % FG::NU, sub = tid / FG::NU;
    const int urow = unit / FG::NCH, uoff = sub < FG::NSUB ? chunk_off(unit % FG::NCH) : -1;
    const int nfr = j1 - j0;
    const int nb = (nfr + fb - 1) / fb;   // slices per stage
    const int nslices = (npr + 3) * nb;   // stages 0 .. npr+2
    const long long fstep = (long long)FG::NSUB * fstride;
    auto issue_slice = [&](int k) {       // one commit group per slice (empty past the last)
        if (k < nslices && uoff >= 0) {
            const int sg = k / nb, f0 = (k - sg * nb) * fb, fn = min(fb, nfr - f0);
            const uint8_t *p = frames + (long long)(j0 + f0 + sub) * fstride +
                               (long long)src_row(2 * sg + urow) * rpitch + uoff;
            uint4 *dst = stg + ((k & 1) * fb + sub) * FG::NU + unit;
            const int fe = PRNU_DCHECK(uoff + 16 <= rowbytes && j0 + f0 + fn <= jmax, uoff) ? fn : 0;
            for (int f = sub; f < fe; f += FG::NSUB, p += fstep, dst += FG::NSUB * FG::NU) cp16(dst, p);
        }
        cp_commit();
    };

    auto stage = [&](int sg) {
        uint32_t ev[4] = {0, 0, 0, 0}, od[4] = {0, 0, 0, 0};
        for (int b = 0; b < nb; ++b) {
            const int k = sg * nb + b;
            issue_slice(k + 1);
            cp_wait_one();  // all but the newest group: slice k has landed
            if (uoff >= 0) {
                const int fn = min(fb, nfr - b * fb);
                const uint4 *src = stg + ((k & 1) * fb + sub) * FG::NU + unit;
                int f = sub;
                // two frames per step: each lane gets both bytes in one three-input add
                for (; f + FG::NSUB < fn; f += 2 * FG::NSUB, src += 2 * FG::NSUB * FG::NU) {
                    const uint4 v = src[0], w = src[FG::NSUB * FG::NU];
                    lanes_add2(v.x, w.x, ev[0], od[0]);
                    lanes_add2(v.y, w.y, ev[1], od[1]);
                    lanes_add2(v.z, w.z, ev[2], od[2]);
                    lanes_add2(v.w, w.w, ev[3], od[3]);
                }
                if (f < fn) {
                    const uint4 v = src[0];
                    lanes_add2(v.x, 0u, ev[0], od[0]);
                    lanes_add2(v.y, 0u, ev[1], od[1]);
                    lanes_add2(v.z, 0u, ev[2], od[2]);
                    lanes_add2(v.w, 0u, ev[3], od[3]);
                }
            }
        }
        if (sub < FG::NSUB) {
            uint4 *pp = reinterpret_cast<uint4 *>(&part[sub][unit][0]);
            pp[0] = make_uint4(ev[0], od[0], ev[1], od[1]);
            pp[1] = make_uint4(ev[2], od[2], ev[3], od[3]);
        }
        __syncthreads();
        // word v of a unit: lanes of bytes b and b + 2, b = 4*(v/2) + v%2 of its chunk
        for (int i = tid; i < FG::NU * 8; i += FG::NT) {
            const int u = i >> 3, v = i & 7;
            uint32_t w = 0;
#pragma unroll
            for (int k = 0; k < FG::NSUB; ++k) w += part[k][u][v];
            const int r = u / FG::NCH, b = 16 * (u % FG::NCH) + 4 * (v >> 1) + (v & 1);
            xs[b % C][r][b / C] = (float)(w & 0xFFFFu);
            xs[(b + 2) % C][r][(b + 2) / C] = (float)(w >> 16);
        }
        __syncthreads();
    };

    // warp (c, g): channel c, output columns cq0 + 32g + lane
    const int c = warp / QG, g = warp % QG;
    const int plane = gi * C + c;
    const bool wact = cq0 + 32 * g < C2;
    const int q = min(cq0 + 32 * g + lane, C2 - 1);  // lanes past the edge recompute the last column
    const bool store_q = wact && cq0 + 32 * g + lane < C2;
    const int px = 2 * (q - cq0);
    const float scale = a.scale_on ? __frcp_rn((float)a.sc.count(plane)) : 1.f;
    float *const X = s.out + (long long)plane * s.H * s.W;
    const int xcol = 2 * cq0 + 64 * g + 2 * lane;  // X columns written by this lane

    // after stage sg: X rows of the strip's own real rows, then the row pass of both rows
    auto consume = [&](int sg, float &h0, float &s0, float &t0, float &h1, float &s1, float &t1) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int t = 2 * sg + r, y = 2 * p0 + t;
            if (t < 2 * npr && y < s.H && xcol < s.W && PRNU_DCHECK(y >= 0, y))
                *reinterpret_cast<float2 *>(X + (long long)y * s.W + xcol) =
                    *reinterpret_cast<const float2 *>(&xs[c][r][64 * g + 2 * lane]);
        }
        float v[8], w[8], rl_;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const float2 *pr = reinterpret_cast<const float2 *>(&xs[c][r][px]);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 u = pr[k];
                v[2 * k] = u.x;
                v[2 * k + 1] = u.y;
            }
            if (r == 0)
                row_math<true>(a.f, v, w, h0, rl_, s0, t0);
            else
                row_math<true>(a.f, v, w, h1, rl_, s1, t1);
        }
    };

    float rh[8], rl[8], rs[8], rt[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) rl[k] = 0.f;
    issue_slice(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {  // input rows 0..5
        stage(k);
        consume(k, rh[2 * k], rs[2 * k], rt[2 * k], rh[2 * k + 1], rs[2 * k + 1], rt[2 * k + 1]);
    }
    for (int i = 0; i < npr; i += 4) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (i + j >= npr) break;  // block-uniform
            // input rows 2p+6, 2p+7 of output row p = p0+i+j go to slots (2j+6) mod 8, (2j+7) mod 8
            const int s6 = (2 * j + 6) & 7, s7 = (2 * j + 7) & 7;
            stage(i + j + 3);
            consume(i + j + 3, rh[s6], rs[s6], rt[s6], rh[s7], rs[s7], rt[s7]);
            const int p = p0 + i + j;
            if (store_q && PRNU_DCHECK(p < R2 && q < C2 && plane < a.P, (long long)p * C2 + q))
                col_store<true, T>(a, rh, rl, rs, rt, (2 * j) & 7, ((long long)plane * R2 + p) * C2 + q, scale);
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");  // no copy outstanding at exit
}

template <int C, int QG, class T>
void launch_t(const SdaArgs &s, const AnaArgs &a, int num_sms, int strips, int max_n, cudaStream_t st) {
    using FG = FusedGeo<C, QG>;
    const int R2 = a.R >> 1, C2 = a.Cc >> 1;
    const int ncb = (C2 + 32 * QG - 1) / (32 * QG);
    if (strips <= 0) {
        // Every block walks its strip at about the same pace, two blocks per SM:
        // the launch takes (waves of blocks) x (stages of a strip, its 3-stage
        // halo included).  Pick the strip count (strips of at least 16 output
        // rows) that minimises that product.
        const long long slots = 2LL * num_sms, base = (long long)ncb * s.G;
        long long best = -1;
        for (int k = 1; k <= std::max(1, R2 / 16); ++k) {
            const long long waves = (base * k + slots - 1) / slots;
            const long long cost = waves * ((R2 + k - 1) / k + 3);
            if (best < 0 || cost < best) {
                best = cost;
                strips = k;
            }
        }
    }
    const int spr = (R2 + strips - 1) / strips;
    const int fb = std::min(max_n, kMaxSlice);
    const size_t smem = (size_t)2 * fb * FG::NU * 16;
    cudaFuncSetAttribute(k_sda_dwt<C, QG, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const dim3 grid((unsigned)ncb, (unsigned)s.G, (unsigned)((R2 + spr - 1) / spr));
    k_sda_dwt<C, QG, T><<<grid, FG::NT, smem, st>>>(s, a, spr, fb);
}

template <class T>
void launch_c(const SdaArgs &s, const AnaArgs &a, int num_sms, int strips, int max_n, cudaStream_t st) {
    if (s.C == 3)
        launch_t<3, 2, T>(s, a, num_sms, strips, max_n, st);
    else
        launch_t<1, 4, T>(s, a, num_sms, strips, max_n, st);
}

}  // namespace

bool sda_dwt_applies(const SdaArgs &s, const AnaArgs &a, const PassDesc *pd) {
    if (s.frame_half || (s.C != 1 && s.C != 3) || (s.gd != nullptr) != (pd != nullptr)) return false;
    if (a.Cc != s.W || a.W != s.W || a.H != s.H || a.R < s.H || a.P != s.G * s.C || (s.W * s.C) % 16 != 0)
        return false;
    auto aligned = [](const uint8_t *f, long long fs, long long rp) {
        return ((reinterpret_cast<uintptr_t>(f) | (uintptr_t)fs | (uintptr_t)rp) & 15u) == 0;
    };
    if (!pd) return s.d >= 1 && s.d <= 257 && aligned(s.frames, s.frame_stride, s.row_pitch);
    if (pd->G != s.G) return false;
    for (int i = 0; i < pd->G; ++i)
        if (pd->g[i].n < 1 || pd->g[i].n > 257 || !aligned(pd->g[i].frames, pd->g[i].frame_stride, pd->g[i].row_pitch))
            return false;
    return true;
}

cudaError_t launch_sda_dwt(const SdaArgs &s, const AnaArgs &a, const PassDesc *pd, int num_sms, cudaStream_t st,
                           int strips) {
    if (!sda_dwt_applies(s, a, pd)) return cudaErrorInvalidValue;
    int max_n = s.d;
    if (pd) {
        max_n = 1;
        for (int i = 0; i < pd->G; ++i) max_n = std::max(max_n, pd->g[i].n);
    }
    if (a.sdt == SB_F16)
        launch_c<__half>(s, a, num_sms, strips, max_n, st);
    else if (a.sdt == SB_BF16)
        launch_c<__nv_bfloat16>(s, a, num_sms, strips, max_n, st);
    else
        launch_c<float>(s, a, num_sms, strips, max_n, st);
    return cudaGetLastError();
}

}  // namespace prnu
