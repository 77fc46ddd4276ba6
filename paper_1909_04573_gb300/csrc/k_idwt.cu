// k_idwt.cu -- inverse DWT of the noise coefficients (synthesis, the
// transpose of the periodised analysis) and the fused level-1 step that forms
// the residual W = I - F(I) = IDWT(0, noise details) (Sec. II-A), crops the
// padding and either stores W or accumulates the MLE sums
// num += W I, den += I^2 (Sec. III-A / III-B).
//
// Gather form of x[(2n+k) mod N] += h[k] a[n] + g[k] b[n]: output sample
// j = 2m + e (e in {0, 1}) takes k = e + 2t, n = m - t for t = 0..3.
// Columns are synthesised first, then rows.  A 32 x 32 output tile needs a
// 19 x 19 tile (3-coefficient halo) of each of the four subbands.
#include <type_traits>

#include "kernels.cuh"

namespace prnu {

constexpr int OT = 32, CT = OT / 2 + 3;  // output tile, coefficient tile
constexpr int NPAIR = OT / 2;              // output pairs per tile row / column

struct SynTile {
    float c[4][CT][CT + 1];
    float lo[OT][CT + 1], hi[OT][CT + 1];
};

// Stage the four coefficient tiles of output tile (y0, x0) of one plane:
// coefficient rows m0-3 .. m0+15 and columns n0-3 .. n0+15 (periodic).
template <class T>
__device__ __forceinline__ void load_coeffs(SynTile &s, const T *LL, const T *LH, const T *HL, const T *HH,
                                            long long poff, int Rc, int Cc, int y0, int x0) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    if (tx < CT && PRNU_DCHECK(wrap_near((x0 >> 1) - 3 + tx, Cc) < Cc, tx)) {
        const int sx = wrap_near((x0 >> 1) - 3 + tx, Cc);
        for (int r = ty; r < CT; r += 8) {
            const long long o = poff + (long long)wrap_near((y0 >> 1) - 3 + r, Rc) * Cc + sx;
            s.c[0][r][tx] = LL ? ldf<T>(LL + o) : 0.f;
            s.c[1][r][tx] = ldf<T>(LH + o);
            s.c[2][r][tx] = ldf<T>(HL + o);
            s.c[3][r][tx] = ldf<T>(HH + o);
        }
    }
}

// Column synthesis: item (coefficient column c, output row pair m) makes
// rows 2m and 2m+1 of lo/hi from coefficient rows m..m+3 of the tile.
__device__ __forceinline__ void synth_cols(SynTile &s, const Filt &f, int tid) {
    for (int it = tid; it < NPAIR * CT; it += 256) {
        const int m = it / CT, c = it - m * CT;
        float a[4], b[4], u[4], v[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            a[t] = s.c[0][m + 3 - t][c];
            b[t] = s.c[1][m + 3 - t][c];
            u[t] = s.c[2][m + 3 - t][c];
            v[t] = s.c[3][m + 3 - t][c];
        }
        float lo0, lo1, hi0, hi1;
        synth_pair2(f, a, b, lo0, lo1);
        synth_pair2(f, u, v, hi0, hi1);
        s.lo[2 * m][c] = lo0;
        s.lo[2 * m + 1][c] = lo1;
        s.hi[2 * m][c] = hi0;
        s.hi[2 * m + 1][c] = hi1;
    }
}

// Row synthesis of the output pair (y, 2n), (y, 2n+1).
__device__ __forceinline__ float2 synth_pair(const SynTile &s, const Filt &f, int y, int n) {
    float l[4], h[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        l[t] = s.lo[y][n + 3 - t];
        h[t] = s.hi[y][n + 3 - t];
    }
    float o0, o1;
    synth_pair2(f, l, h, o0, o1);
    return make_float2(o0, o1);
}

template <class T>
__global__ void __launch_bounds__(256) k_synthesis(SynArgs a) {
    __shared__ SynTile s;
    const int plane = blockIdx.z;
    const int y0 = blockIdx.y * OT, x0 = blockIdx.x * OT;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const long long poff = (long long)plane * a.Rc * a.Cc;
    load_coeffs<T>(s, static_cast<const T *>(a.LL), static_cast<const T *>(a.LH), static_cast<const T *>(a.HL),
                   static_cast<const T *>(a.HH), poff, a.Rc, a.Cc, y0, x0);
    __syncthreads();
    synth_cols(s, a.f, tid);
    __syncthreads();
    const int Ro = 2 * a.Rc, Co = 2 * a.Cc;  // even, so a pair is in range or out together
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int it = tid + 256 * k;
        const int y = it >> 4, n = it & 15;
        const int gy = y0 + y, gx = x0 + 2 * n;
        if (gy < Ro && gx < Co) {
            const float2 v = synth_pair(s, a.f, y, n);
            T *o = static_cast<T *>(a.out) + ((long long)plane * Ro + gy) * Co + gx;
            stf<T>(o, v.x);
            stf<T>(o + 1, v.y);
        }
    }
}

// Level 1: W for the cropped H x W region.  Residual mode: one plane per
// grid z, W stored at res_out[plane].  MLE mode: grid z is the channel and
// the block walks the pass's G images, summing W*I and I*I in registers
// before one read-modify-write of num/den.
// Add a thread's 4 MLE sums (plain or float-float pairs) into num/den.
template <bool COMP>
__device__ __forceinline__ void mle_flush(const FinalArgs &a, float *num, float *den, float *an, float *ad,
                                          float *anl, float *adl, int y0, int x0, int tid) {
    const long long hw = (long long)a.H * a.W;
    const long long chw = (long long)a.C * hw;  // offset of the low parts when COMP
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int it = tid + 256 * k;
        const int y = it >> 4, n = it & 15;
        const int gy = y0 + y, gx = x0 + 2 * n;
        if (gy >= a.H || gx >= a.W) continue;
        const long long o = (long long)blockIdx.z * hw + (long long)gy * a.W + gx;
        const int cnt = PRNU_DCHECK((int)blockIdx.z < a.C, blockIdx.z) ? (gx + 1 < a.W ? 2 : 1) : 0;
        for (int e = 0; e < cnt; ++e) {
            const int j = 2 * k + e;
            if (COMP) {
                float h = num[o + e], l = num[chw + o + e];
                ff_add(h, l, an[j]);
                l = __fadd_rn(l, anl[j]);
                num[o + e] = h;
                num[chw + o + e] = l;
                h = den[o + e];
                l = den[chw + o + e];
                ff_add(h, l, ad[j]);
                l = __fadd_rn(l, adl[j]);
                den[o + e] = h;
                den[chw + o + e] = l;
            } else {
                num[o + e] += an[j];
                den[o + e] += ad[j];
            }
        }
    }
}

template <bool MLE, class T, bool COMP>
__global__ void __launch_bounds__(256) k_final(FinalArgs a) {
    __shared__ SynTile s;
    const int y0 = blockIdx.y * OT, x0 = blockIdx.x * OT;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    // MLE sums of the 4 outputs this thread owns; with COMP a float-float
    // pair each (compensated summation across the pass's images)
    float an[4], ad[4], anl[4], adl[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) { an[k] = 0.f; ad[k] = 0.f; anl[k] = 0.f; adl[k] = 0.f; }
    const long long hw = (long long)a.H * a.W;
    const int nimg = MLE ? a.G : 1;
    int cam = a.gd ? a.gd[0].cam : -1;  // multi-camera pass: current camera
    for (int i = 0; i < nimg; ++i) {
        const int plane = MLE ? i * a.C + (int)blockIdx.z : (int)blockIdx.z;
        if (a.gd && a.gd[i].cam != cam) {  // block-uniform: the camera changes
            mle_flush<COMP>(a, a.cams[cam].num, a.cams[cam].den, an, ad, anl, adl, y0, x0, tid);
#pragma unroll
            for (int k = 0; k < 4; ++k) { an[k] = 0.f; ad[k] = 0.f; anl[k] = 0.f; adl[k] = 0.f; }
            cam = a.gd[i].cam;
        }
        const long long poff = (long long)plane * a.Rc * a.Cc;
        if (i > 0) __syncthreads();
        load_coeffs<T>(s, static_cast<const T *>(a.LL), static_cast<const T *>(a.LH), static_cast<const T *>(a.HL),
                       static_cast<const T *>(a.HH), poff, a.Rc, a.Cc, y0, x0);
        __syncthreads();
        synth_cols(s, a.f, tid);
        __syncthreads();
        const float inv_n = __frcp_rn((float)a.sc.count(plane));
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int it = tid + 256 * k;
            const int y = it >> 4, n = it & 15;
            const int gy = y0 + y, gx = x0 + 2 * n;
            if (gy >= a.H || gx >= a.W) continue;
            const float2 w = synth_pair(s, a.f, y, n);
            const long long o = (long long)plane * hw + (long long)gy * a.W + gx;
            const bool two = gx + 1 < a.W;
            if (MLE) {
                const float I0 = __ldg(a.X + o) * inv_n;
                const float I1 = two ? __ldg(a.X + o + 1) * inv_n : 0.f;
                if (COMP) {
                    ff_add(an[2 * k], anl[2 * k], w.x * I0);
                    ff_add(ad[2 * k], adl[2 * k], I0 * I0);
                    if (two) {
                        ff_add(an[2 * k + 1], anl[2 * k + 1], w.y * I1);
                        ff_add(ad[2 * k + 1], adl[2 * k + 1], I1 * I1);
                    }
                } else {
                    an[2 * k] = __fmaf_rn(w.x, I0, an[2 * k]);
                    ad[2 * k] = __fmaf_rn(I0, I0, ad[2 * k]);
                    if (two) {
                        an[2 * k + 1] = __fmaf_rn(w.y, I1, an[2 * k + 1]);
                        ad[2 * k + 1] = __fmaf_rn(I1, I1, ad[2 * k + 1]);
                    }
                }
            } else {
                if (a.accumulate) {
                    a.res_out[o] += w.x;
                    if (two) a.res_out[o + 1] += w.y;
                } else {
                    a.res_out[o] = w.x;
                    if (two) a.res_out[o + 1] = w.y;
                }
            }
        }
    }
    if (MLE) {
        if (a.gd)
            mle_flush<COMP>(a, a.cams[cam].num, a.cams[cam].den, an, ad, anl, adl, y0, x0, tid);
        else
            mle_flush<COMP>(a, a.num, a.den, an, ad, anl, adl, y0, x0, tid);
    }
}


// ---------------------------------------------------------------------------
// MLE mode with float32 subbands: the same level-1 step as k_final with the
// coefficient tiles and image tile of the next two images fetched by cp.async
// into two more buffers while the current image is synthesised (a tile's
// synthesis is too short to cover one copy latency).
//
// Staging moves 16-byte chunks: a coefficient tile row is the 24 columns
// n0-4 .. n0+19 (n0 = x0/2; the synthesis reads n0-3 .. n0+15), which start on
// a 4-float boundary, and since the coefficient width Cc is a multiple of 8 a
// periodic wrap never splits a chunk; image tile rows are 8 chunks (a ragged
// right edge or a width that is not a multiple of 4 falls back to 4-byte
// copies).  The column pass gives warp w the output row pairs of coefficient
// rows 2w, 2w+1 with one coefficient column per lane (lanes 0..18), so its
// shared-memory reads and writes are consecutive in a row; lo and hi share
// rows of 48 floats (hi at +24), so the two output rows a warp reads in the
// row pass sit 16 banks apart.

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

constexpr int AC_W = 24;   // lo | hi split of a row of lh
constexpr int AC_LH = 48;  // lo | hi row: lo at 0..18, hi at 24..42
constexpr int AC_BUF = 3;  // copy stages
// Staged coefficient columns per tile row for subband type T: float32 rows
// are columns n0-4 .. n0+19 (6 chunks of 4), 16-bit rows n0-8 .. n0+23 (4
// chunks of 8); the synthesis reads n0-3 .. n0+15 at offset ACOFF.
template <class T> struct ACT {
    static constexpr int EPC = 16 / (int)sizeof(T);        // elements per 16-byte chunk
    static constexpr int W = sizeof(T) == 4 ? 24 : 32;     // staged columns
    static constexpr int CPR = W / EPC;                    // chunks per row
    static constexpr int START = sizeof(T) == 4 ? 4 : 8;   // first staged column is n0 - START
    static constexpr int OFF = START - 3;                  // column of n0 - 3 in the staged row
};
template <class T>
struct AsyncTile {
    T c[AC_BUF][4][CT][ACT<T>::W];  // LL, LH, HL, HH coefficient tiles
    float x[AC_BUF][OT][OT];        // the image tile (group sums)
    float lh[OT][AC_LH];            // column-synthesised lo (0..18) and hi (24..42)
};

template <bool COMP, class T>
__global__ void __launch_bounds__(256, 5) k_final_async(FinalArgs a) {
    using At = ACT<T>;
    __shared__ __align__(16) AsyncTile<T> s;
    const int y0 = blockIdx.y * OT, x0 = blockIdx.x * OT;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * 32 + tx;
    const long long hw = (long long)a.H * a.W;
    const T *LL = static_cast<const T *>(a.LL), *LH = static_cast<const T *>(a.LH);
    const T *HL = static_cast<const T *>(a.HL), *HH = static_cast<const T *>(a.HH);
    const int nimg = a.G;
    auto plane_of = [&](int i) { return i * a.C + (int)blockIdx.z; };
    // image tile: full 16-byte chunks when the tile's rows are whole chunks
    const bool x16 = (a.W & 3) == 0 && x0 + OT <= a.W && (reinterpret_cast<uintptr_t>(a.X) & 15u) == 0;
    // The copies of every image have the same in-plane offsets: each thread's
    // (at most two) coefficient chunks -- subband k, row, 4-column group -- and
    // its image chunk are resolved once, so an image's issue is a handful of
    // adds per copy.
    constexpr int NCH = 4 * CT * At::CPR;  // coefficient chunks (456 float32, 304 16-bit)
    int ck[2], coff[2], cdst[2];           // subband (-1: none), in-plane offset, element index in s.c[0]
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int it = tid + 256 * h;
        ck[h] = -1;
        coff[h] = 0;
        cdst[h] = 0;
        if (it < NCH) {
            const int k = it / (CT * At::CPR), rem = it - k * (CT * At::CPR);
            const int r = rem / At::CPR, j = rem - r * At::CPR;
            const int row = wrap_near((y0 >> 1) - 3 + r, a.Rc);
            const int col = wrap_near((x0 >> 1) - At::START + At::EPC * j, a.Cc);
            if (PRNU_DCHECK(row >= 0 && row < a.Rc && col >= 0 && col + At::EPC - 1 < a.Cc, col)) {
                ck[h] = k;
                coff[h] = row * a.Cc + col;
                cdst[h] = (k * CT + r) * At::W + At::EPC * j;
            }
        }
    }
    const int xy = tid >> 3, xj = tid & 7;  // x16: 32 rows x 8 chunks
    const bool xrow = y0 + xy < a.H && PRNU_DCHECK(!x16 || x0 + 4 * xj + 3 < a.W, x0 + 4 * xj);
    const long long xoff = (long long)(y0 + xy) * a.W + x0 + 4 * xj;
    auto issue = [&](int plane, int b) {
        const long long poff = (long long)plane * a.Rc * a.Cc;
        T *cb = &s.c[b][0][0][0];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (ck[h] < 0) continue;
            const T *src = ck[h] == 0 ? LL : ck[h] == 1 ? LH : ck[h] == 2 ? HL : HH;
            if (src)
                cp_async16(cb + cdst[h], src + poff + coff[h]);
            else
                *reinterpret_cast<float4 *>(cb + cdst[h]) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const float *xp = a.X + (long long)plane * hw;
        if (x16) {
            if (xrow) cp_async16(&s.x[b][xy][4 * xj], xp + xoff);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int it = tid + 256 * k;
                const int y = it >> 5, xx = it & 31;
                const int gy = y0 + y, gx = x0 + xx;
                if (gy < a.H && gx < a.W) cp_async4(&s.x[b][y][xx], xp + (long long)gy * a.W + gx);
            }
        }
    };
    float an[4], ad[4], anl[4], adl[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) { an[k] = 0.f; ad[k] = 0.f; anl[k] = 0.f; adl[k] = 0.f; }
    int cam = a.gd ? a.gd[0].cam : -1;
    issue(plane_of(0), 0);
    cp_commit();
    if (nimg > 1) issue(plane_of(1), 1);
    cp_commit();  // one group per image slot, empty past the last image
    for (int i = 0; i < nimg; ++i) {
        const int b = i % AC_BUF;
        const int plane = plane_of(i);
        cp_wait_one();
        __syncthreads();  // image i landed; every reader of image i-1's buffer and of lh is done
        if (i + 2 < nimg) issue(plane_of(i + 2), (i + 2) % AC_BUF);
        cp_commit();
        if (a.gd && a.gd[i].cam != cam) {  // block-uniform: the camera changes
            mle_flush<COMP>(a, a.cams[cam].num, a.cams[cam].den, an, ad, anl, adl, y0, x0, tid);
#pragma unroll
            for (int k = 0; k < 4; ++k) { an[k] = 0.f; ad[k] = 0.f; anl[k] = 0.f; adl[k] = 0.f; }
            cam = a.gd[i].cam;
        }
        // column synthesis from buffer b: warp ty owns coefficient rows
        // m = 2ty, 2ty+1 (output rows 4ty .. 4ty+3), which read tile rows
        // 2ty .. 2ty+4 (each loaded once), lane tx one coefficient column
        if (tx < CT) {
            float q[5][4];  // [tile row - 2ty][subband]
#pragma unroll
            for (int rr = 0; rr < 5; ++rr)
#pragma unroll
                for (int k = 0; k < 4; ++k) q[rr][k] = to_f(s.c[b][k][2 * ty + rr][tx + At::OFF]);
#pragma unroll
            for (int mm = 0; mm < 2; ++mm) {
                const int m = 2 * ty + mm;
                float c0[4], c1[4], c2[4], c3[4];  // coefficient row m - t is tile row m + 3 - t
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    c0[t] = q[mm + 3 - t][0];
                    c1[t] = q[mm + 3 - t][1];
                    c2[t] = q[mm + 3 - t][2];
                    c3[t] = q[mm + 3 - t][3];
                }
                float lo0, lo1, hi0, hi1;
                synth_pair2(a.f, c0, c1, lo0, lo1);
                synth_pair2(a.f, c2, c3, hi0, hi1);
                s.lh[2 * m][tx] = lo0;
                s.lh[2 * m + 1][tx] = lo1;
                s.lh[2 * m][AC_W + tx] = hi0;
                s.lh[2 * m + 1][AC_W + tx] = hi1;
            }
        }
        __syncthreads();
        const float inv_n = __frcp_rn((float)a.sc.count(plane));
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int it = tid + 256 * k;
            const int y = it >> 4, n = it & 15;
            const int gy = y0 + y, gx = x0 + 2 * n;
            if (gy >= a.H || gx >= a.W) continue;
            const bool two = gx + 1 < a.W;
            float l[4], h[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                l[t] = s.lh[y][n + 3 - t];
                h[t] = s.lh[y][AC_W + n + 3 - t];
            }
            float w[2];
            synth_pair2(a.f, l, h, w[0], w[1]);
            const float2 xv = *reinterpret_cast<const float2 *>(&s.x[b][y][2 * n]);
            const float I0 = xv.x * inv_n;
            const float I1 = two ? xv.y * inv_n : 0.f;
            if (COMP) {
                ff_add(an[2 * k], anl[2 * k], w[0] * I0);
                ff_add(ad[2 * k], adl[2 * k], I0 * I0);
                if (two) {
                    ff_add(an[2 * k + 1], anl[2 * k + 1], w[1] * I1);
                    ff_add(ad[2 * k + 1], adl[2 * k + 1], I1 * I1);
                }
            } else {
                an[2 * k] = __fmaf_rn(w[0], I0, an[2 * k]);
                ad[2 * k] = __fmaf_rn(I0, I0, ad[2 * k]);
                if (two) {
                    an[2 * k + 1] = __fmaf_rn(w[1], I1, an[2 * k + 1]);
                    ad[2 * k + 1] = __fmaf_rn(I1, I1, ad[2 * k + 1]);
                }
            }
        }
    }
    cp_wait_all();  // no copy in flight at exit (the trailing groups are empty)
    if (a.gd)
        mle_flush<COMP>(a, a.cams[cam].num, a.cams[cam].den, an, ad, anl, adl, y0, x0, tid);
    else
        mle_flush<COMP>(a, a.num, a.den, an, ad, anl, adl, y0, x0, tid);
}


// Wide-tile form of the MLE step for float32 subbands: a 58 x 32 output tile
// needs exactly 32 coefficient columns (29 + the 3-column halo), one per
// lane, so the column synthesis keeps every lane busy (the 32 x 32 tile's 19
// columns leave 13 of 32 idle); in the row synthesis warp w takes output rows
// 4w .. 4w+3 and lane n the output pair 2n, 2n+1 (29 of 32 lanes).  The
// copies of image i+2 are in flight while image i is synthesised, as in
// k_final_async, and every output takes the same operations in the same order
// (column synthesis, row synthesis, then W I and I I image by image), so the
// sums are identical.  Needs W even, Cc a multiple of 4, 16-byte aligned
// subbands and 8-byte aligned group sums (the launcher checks).
constexpr int AW_OW = 58, AW_OH = 32;  // output tile
constexpr int AW_PAIRS = AW_OW / 2;    // output pairs per tile row
constexpr int AW_CW = 32, AW_CH = 19;  // coefficient tile: columns n0-3 .. n0+28, rows m0-3 .. m0+15
constexpr int AW_SW = 36;              // staged columns: 9 aligned 4-column chunks from (n0-3) rounded down
template <int BUF>
struct AsyncTileW {
    float c[BUF][4][AW_CH][AW_SW];  // LL, LH, HL, HH
    float x[BUF][AW_OH][AW_OW];     // the image tile (group sums)
    float lh[AW_OH][2 * AW_CW];     // column-synthesised lo (0..31) and hi (32..63)
};

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}

template <bool COMP, int BUF>
__global__ void __launch_bounds__(256, BUF == 2 ? 4 : 3) k_final_async_w(FinalArgs a) {
    extern __shared__ __align__(16) unsigned char aw_smem[];
    AsyncTileW<BUF> &s = *reinterpret_cast<AsyncTileW<BUF> *>(aw_smem);
    const int y0 = blockIdx.y * AW_OH, x0 = blockIdx.x * AW_OW;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long hw = (long long)a.H * a.W;
    const float *LL = static_cast<const float *>(a.LL), *LH = static_cast<const float *>(a.LH);
    const float *HL = static_cast<const float *>(a.HL), *HH = static_cast<const float *>(a.HH);
    const int nimg = a.G;
    auto plane_of = [&](int i) { return i * a.C + (int)blockIdx.z; };
    const int n0 = x0 >> 1, m0 = y0 >> 1;
    const int cs = (n0 - 3) & ~3;    // first staged column (a multiple of 4; -4 for the first tile)
    const int coff0 = (n0 - 3) - cs;  // staged column of n0 - 3
    // each thread's (at most three) coefficient chunks -- subband, row, chunk -- and
    // (at most four) image pairs, resolved once: an image's issue is a few adds per copy
    constexpr int NCH = 4 * AW_CH * (AW_SW / 4);  // 684
    int ck[3], coff[3], cdst[3];
#pragma unroll
    for (int h = 0; h < 3; ++h) {
        const int it = tid + 256 * h;
        ck[h] = -1;
        coff[h] = 0;
        cdst[h] = 0;
        if (it < NCH) {
            const int k = it / (AW_CH * (AW_SW / 4)), rem = it - k * (AW_CH * (AW_SW / 4));
            const int r = rem / (AW_SW / 4), j = rem - r * (AW_SW / 4);
            const int row = wrap_near(m0 - 3 + r, a.Rc);
            const int col = wrap_near(cs + 4 * j, a.Cc);
            if (PRNU_DCHECK(row >= 0 && row < a.Rc && col >= 0 && col + 3 < a.Cc, col)) {
                ck[h] = k;
                coff[h] = row * a.Cc + col;
                cdst[h] = (k * AW_CH + r) * AW_SW + 4 * j;
            }
        }
    }
    long long xoff[4];
    int xdst[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const int it = tid + 256 * h;
        xdst[h] = -1;
        xoff[h] = 0;
        if (it < AW_OH * AW_PAIRS) {
            const int yy = it / AW_PAIRS, pp = it - yy * AW_PAIRS;
            const int gy = y0 + yy, gx = x0 + 2 * pp;
            if (gy < a.H && PRNU_DCHECK(gx + 1 < a.W || gx >= a.W, gx) && gx < a.W) {
                xdst[h] = yy * AW_OW + 2 * pp;
                xoff[h] = (long long)gy * a.W + gx;
            }
        }
    }
    auto issue = [&](int plane, int b) {
        const long long poff = (long long)plane * a.Rc * a.Cc;
        float *cb = &s.c[b][0][0][0];
#pragma unroll
        for (int h = 0; h < 3; ++h) {
            if (ck[h] < 0) continue;
            const float *src = ck[h] == 0 ? LL : ck[h] == 1 ? LH : ck[h] == 2 ? HL : HH;
            if (src)
                cp_async16(cb + cdst[h], src + poff + coff[h]);
            else
                *reinterpret_cast<float4 *>(cb + cdst[h]) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const float *xp = a.X + (long long)plane * hw;
        float *xb = &s.x[b][0][0];
#pragma unroll
        for (int h = 0; h < 4; ++h)
            if (xdst[h] >= 0) cp_async8(xb + xdst[h], xp + xoff[h]);
    };
    float an[4][2], ad[4][2], anl[4][2], adl[4][2];  // [output row 4w + r][column 2n + c]
    auto reset = [&] {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                an[r][c] = 0.f;
                ad[r][c] = 0.f;
                anl[r][c] = 0.f;
                adl[r][c] = 0.f;
            }
    };
    // add the thread's sums into num/den (float-float pairs with COMP)
    auto flush = [&](float *num, float *den) {
        if (lane >= AW_PAIRS) return;
        const long long chw = (long long)a.C * hw;  // offset of the low parts when COMP
        const int gx = x0 + 2 * lane;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int gy = y0 + 4 * warp + r;
            if (gy >= a.H || gx >= a.W || !PRNU_DCHECK((int)blockIdx.z < a.C, blockIdx.z)) continue;
            const long long o = (long long)blockIdx.z * hw + (long long)gy * a.W + gx;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (COMP) {
                    float h = num[o + c], l = num[chw + o + c];
                    ff_add(h, l, an[r][c]);
                    l = __fadd_rn(l, anl[r][c]);
                    num[o + c] = h;
                    num[chw + o + c] = l;
                    h = den[o + c];
                    l = den[chw + o + c];
                    ff_add(h, l, ad[r][c]);
                    l = __fadd_rn(l, adl[r][c]);
                    den[o + c] = h;
                    den[chw + o + c] = l;
                } else {
                    num[o + c] += an[r][c];
                    den[o + c] += ad[r][c];
                }
            }
        }
    };
    reset();
    int cam = a.gd ? a.gd[0].cam : -1;
    // BUF == 3: images i+1 and i+2 in flight while image i is synthesised;
    // BUF == 2: image i+1
    issue(plane_of(0), 0);
    cp_commit();
    if (BUF == 3) {
        if (nimg > 1) issue(plane_of(1), 1);
        cp_commit();  // one group per image slot, empty past the last image
    }
    for (int i = 0; i < nimg; ++i) {
        const int b = i % BUF;
        const int plane = plane_of(i);
        if (BUF == 2) {
            cp_wait_all();    // image i landed
            __syncthreads();  // every reader of image i-1's buffer and of lh is done
            if (i + 1 < nimg) issue(plane_of(i + 1), (i + 1) % BUF);
            cp_commit();
        } else {
            cp_wait_one();
            __syncthreads();  // image i landed; every reader of image i-1's buffer and of lh is done
            if (i + 2 < nimg) issue(plane_of(i + 2), (i + 2) % BUF);
            cp_commit();
        }
        if (a.gd && a.gd[i].cam != cam) {  // block-uniform: the camera changes
            flush(a.cams[cam].num, a.cams[cam].den);
            reset();
            cam = a.gd[i].cam;
        }
        // column synthesis from buffer b: warp w owns coefficient rows m = 2w, 2w+1
        // (output rows 4w .. 4w+3), which read tile rows 2w .. 2w+4; lane = tile column
        {
            float q[5][4];  // [tile row - 2w][subband]
#pragma unroll
            for (int rr = 0; rr < 5; ++rr)
#pragma unroll
                for (int k = 0; k < 4; ++k) q[rr][k] = s.c[b][k][2 * warp + rr][lane + coff0];
#pragma unroll
            for (int mm = 0; mm < 2; ++mm) {
                const int m = 2 * warp + mm;
                float c0[4], c1[4], c2[4], c3[4];  // coefficient row m - t is tile row m + 3 - t
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    c0[t] = q[mm + 3 - t][0];
                    c1[t] = q[mm + 3 - t][1];
                    c2[t] = q[mm + 3 - t][2];
                    c3[t] = q[mm + 3 - t][3];
                }
                float lo0, lo1, hi0, hi1;
                synth_pair2(a.f, c0, c1, lo0, lo1);
                synth_pair2(a.f, c2, c3, hi0, hi1);
                s.lh[2 * m][lane] = lo0;
                s.lh[2 * m + 1][lane] = lo1;
                s.lh[2 * m][AW_CW + lane] = hi0;
                s.lh[2 * m + 1][AW_CW + lane] = hi1;
            }
        }
        __syncthreads();
        const float inv_n = __frcp_rn((float)a.sc.count(plane));
        if (lane < AW_PAIRS) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int y = 4 * warp + r;
                const int gy = y0 + y, gx = x0 + 2 * lane;
                if (gy >= a.H || gx >= a.W) continue;
                float l[4], h[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    l[t] = s.lh[y][lane + 3 - t];
                    h[t] = s.lh[y][AW_CW + lane + 3 - t];
                }
                float w[2];
                synth_pair2(a.f, l, h, w[0], w[1]);
                const float2 xv = *reinterpret_cast<const float2 *>(&s.x[b][y][2 * lane]);
                const float I0 = xv.x * inv_n, I1 = xv.y * inv_n;
                if (COMP) {
                    ff_add(an[r][0], anl[r][0], w[0] * I0);
                    ff_add(ad[r][0], adl[r][0], I0 * I0);
                    ff_add(an[r][1], anl[r][1], w[1] * I1);
                    ff_add(ad[r][1], adl[r][1], I1 * I1);
                } else {
                    an[r][0] = __fmaf_rn(w[0], I0, an[r][0]);
                    ad[r][0] = __fmaf_rn(I0, I0, ad[r][0]);
                    an[r][1] = __fmaf_rn(w[1], I1, an[r][1]);
                    ad[r][1] = __fmaf_rn(I1, I1, ad[r][1]);
                }
            }
        }
    }
    cp_wait_all();  // no copy in flight at exit (the trailing groups are empty)
    if (a.gd)
        flush(a.cams[cam].num, a.cams[cam].den);
    else
        flush(a.num, a.den);
}

// ---------------------------------------------------------------------------
// Residual mode with float32 subbands, streaming: a warp owns 32 coefficient
// columns n0 .. n0+31 of one plane and walks a strip of coefficient rows,
// keeping the last four rows of the four subbands in a register ring for the
// column synthesis; the loads of the next coefficient row (and the
// epilogue's inputs of this row, where it has any) are issued before this
// row's arithmetic, so their latency overlaps it.  Lanes 3..31 produce output columns 2n, 2n+1; lanes 0..2
// only supply the row synthesis' left neighbours (taken with shuffles), so
// consecutive warps start 29 columns apart.  Three rows above the strip prime
// the ring.
constexpr int FS_ROWS = 32;  // coefficient rows per strip (64 output rows)
constexpr int FS_WARPS = 4;
constexpr int FS_COLS = 29;  // output coefficient columns per warp

// One warp's strip: coefficient planes [Rc][Cc] (LL may be null: zero).
// With GRAY3 each detail value is 0.299 / 0.587 / 0.114 of the planes at
// offsets 0, cs, 2 cs (the synthesis is linear, so this synthesises the grey
// combination of three channels' noise).  Each output pair (y, x), (y, x+1)
// of the first outH x outW samples goes to epi(y, x, w0, w1, two).
template <bool GRAY3, class T, class Epi>
__device__ __forceinline__ void stream_synth(const T *LL, const T *LH, const T *HL, const T *HH, long long cs, int Rc,
                                             int Cc, const Filt &f, int cg, int m0, int outH, int outW, Epi &epi) {
    const int lane = threadIdx.x & 31;
    const int n = cg * FS_COLS - 3 + lane;  // coefficient column (unwrapped)
    const int nw = wrap_near(n, Cc);
    const bool out_lane = lane >= 3 && n < Cc;
    const int m1 = min(Rc, m0 + FS_ROWS);
    // ring slot of coefficient row m is (m - m0 + 3) & 3
    float q[4][4];  // [slot][subband]
    // raw loads of one coefficient row (LL, then each detail subband's one or
    // three channel values), fetched one row ahead of their use
    constexpr int NR = GRAY3 ? 10 : 4;
    auto fetch = [&](int m, float *r) {
        const long long o = PRNU_DCHECK(nw >= 0 && nw < Cc, nw) ? (long long)wrap_near(m, Rc) * Cc + nw : 0;
        r[0] = LL ? ldf<T>(LL + o) : 0.f;
        const T *sb[3] = {LH, HL, HH};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (GRAY3) {
                r[1 + 3 * k] = ldf<T>(sb[k] + o);
                r[2 + 3 * k] = ldf<T>(sb[k] + o + cs);
                r[3 + 3 * k] = ldf<T>(sb[k] + o + 2 * cs);
            } else {
                r[1 + k] = ldf<T>(sb[k] + o);
            }
        }
    };
    auto combine = [&](const float *r, float *d) {
        d[0] = r[0];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            d[1 + k] = GRAY3 ? __fmaf_rn(0.114f, r[3 + 3 * k], __fmaf_rn(0.587f, r[2 + 3 * k], 0.299f * r[1 + 3 * k]))
                             : r[1 + k];
    };
    float nx[NR];
#pragma unroll
    for (int t = 1; t <= 3; ++t) {
        fetch(m0 - t, nx);
        combine(nx, q[(3 - t) & 3]);
    }
    fetch(m0, nx);
    for (int mb = m0; mb < m1; mb += 4) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = mb + j;
            if (m >= m1) break;
            combine(nx, q[(j + 3) & 3]);
            if (m + 1 < m1) fetch(m + 1, nx);  // the next row's loads overlap this row's synthesis
            epi.prefetch(2 * m, 2 * n, out_lane, outH, outW);  // the epilogue's inputs, beside them
            // column synthesis: rows 2m + e of lo (LL, LH) and hi (HL, HH)
            float lo[2], hi[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                float l = 0.f, h = 0.f;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const float *r = q[(j + 3 - t) & 3];
                    const float hk = f.h[e + 2 * t], gk = f.g[e + 2 * t];
                    l = __fmaf_rn(hk, r[0], l);
                    l = __fmaf_rn(gk, r[1], l);
                    h = __fmaf_rn(hk, r[2], h);
                    h = __fmaf_rn(gk, r[3], h);
                }
                lo[e] = l;
                hi[e] = h;
            }
            // row synthesis of output rows 2m + e, columns 2n + f
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                float L[4], Hh[4];
                L[0] = lo[e];
                Hh[0] = hi[e];
#pragma unroll
                for (int t = 1; t < 4; ++t) {
                    L[t] = __shfl_up_sync(0xffffffffu, lo[e], t);
                    Hh[t] = __shfl_up_sync(0xffffffffu, hi[e], t);
                }
                float w[2];
                synth_pair2(f, L, Hh, w[0], w[1]);
                const int y = 2 * m + e, x = 2 * n;
                if (out_lane && y < outH && x < outW) epi(y, x, w[0], w[1], x + 1 < outW);
            }
        }
    }
}

// store (ACC: add) an output pair into a row-major plane of width W of type T
template <bool ACC, class T = float>
struct StoreEpi {
    T *p;
    int W;
    __device__ __forceinline__ void prefetch(int, int, bool, int, int) {}
    __device__ __forceinline__ void operator()(int y, int x, float w0, float w1, bool two) const {
        T *o = p + (long long)y * W + x;
        if (ACC) {
            stf<T>(o, to_f(o[0]) + w0);
            if (two) stf<T>(o + 1, to_f(o[1]) + w1);
        } else if (std::is_same<T, float>::value && two && ((reinterpret_cast<uintptr_t>(o) & 7u) == 0)) {
            *reinterpret_cast<float2 *>(o) = make_float2(w0, w1);
        } else {
            stf<T>(o, w0);
            if (two) stf<T>(o + 1, w1);
        }
    }
};

// Level 1, residual mode: W cropped to H x W, stored (ACC: added) at res_out[plane].
template <bool ACC, class T>
__global__ void __launch_bounds__(32 * FS_WARPS) k_final_stream(FinalArgs a) {
    const int cg = blockIdx.x * FS_WARPS + (threadIdx.x >> 5);
    if (cg * FS_COLS >= a.Cc) return;  // warp-uniform
    const long long off = (long long)blockIdx.z * a.Rc * a.Cc;
    const T *LL = a.LL ? static_cast<const T *>(a.LL) + off : nullptr;
    StoreEpi<ACC> epi{a.res_out + (long long)blockIdx.z * a.H * a.W, a.W};
    stream_synth<false, T>(LL, static_cast<const T *>(a.LH) + off, static_cast<const T *>(a.HL) + off,
                           static_cast<const T *>(a.HH) + off, 0, a.Rc, a.Cc, a.f, cg, blockIdx.y * FS_ROWS, a.H,
                           a.W, epi);
}

// Levels 2..L: the 2Rc x 2Cc noise LL of the level below (grey with gray3).
template <bool GRAY3, class T>
__global__ void __launch_bounds__(32 * FS_WARPS) k_synthesis_stream(SynArgs a) {
    const int cg = blockIdx.x * FS_WARPS + (threadIdx.x >> 5);
    if (cg * FS_COLS >= a.Cc) return;  // warp-uniform
    const long long A = (long long)a.Rc * a.Cc;
    const long long off = (long long)blockIdx.z * A, doff = GRAY3 ? 3 * off : off;
    const T *LL = a.LL ? static_cast<const T *>(a.LL) + off : nullptr;
    StoreEpi<false, T> epi{static_cast<T *>(a.out) + 4 * off, 2 * a.Cc};
    stream_synth<GRAY3, T>(LL, static_cast<const T *>(a.LH) + doff, static_cast<const T *>(a.HL) + doff,
                           static_cast<const T *>(a.HH) + doff, A, a.Rc, a.Cc, a.f, cg, blockIdx.y * FS_ROWS,
                           2 * a.Rc, 2 * a.Cc, epi);
}

// Level 1, PCE mode: X = grey W, Y = K grey(I), and the lane's sums of X,
// X^2, Y, Y^2 as float-float pairs (no float64 arithmetic per pixel).
struct PceEpi {
    float *X, *Y;
    const float *K, *I;
    long long hw;
    int W, C;
    bool vec;  // W even and every base 8-byte aligned: pairs move as float2
    float m[4] = {0.f, 0.f, 0.f, 0.f}, mlo[4] = {0.f, 0.f, 0.f, 0.f};
    float2 pi[2][3], pk[2];  // output rows 2m, 2m+1: image channels and K at (y, x), (y, x+1)
    __device__ __forceinline__ float2 ld2(const float *p, bool two) const {
        if (vec && two) return __ldg(reinterpret_cast<const float2 *>(p));
        return make_float2(__ldg(p), two ? __ldg(p + 1) : 0.f);
    }
    __device__ __forceinline__ void st2(float *p, float a, float b, bool two) const {
        if (vec && two) {
            *reinterpret_cast<float2 *>(p) = make_float2(a, b);
        } else {
            p[0] = a;
            if (two) p[1] = b;
        }
    }
    // loads of output rows y0, y0+1 at columns x, x+1, issued one coefficient
    // row ahead of their use so their latency overlaps the synthesis
    __device__ __forceinline__ void prefetch(int y0, int x, bool lane_ok, int outH, int outW) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int y = y0 + e;
            if (lane_ok && y < outH && x < outW) {
                const bool two = x + 1 < outW;
                const long long o = (long long)y * W + x;
                pi[e][0] = ld2(I + o, two);
                if (C == 3) {
                    pi[e][1] = ld2(I + hw + o, two);
                    pi[e][2] = ld2(I + 2 * hw + o, two);
                }
                pk[e] = ld2(K + o, two);
            }
        }
    }
    __device__ __forceinline__ void operator()(int y, int x, float w0, float w1, bool two) {
        const long long o = (long long)y * W + x;
        const int e = y & 1;
        float2 g = pi[e][0];
        if (C == 3) {
            const float2 i1 = pi[e][1], i2 = pi[e][2];
            g.x = __fmaf_rn(0.114f, i2.x, __fmaf_rn(0.587f, i1.x, 0.299f * g.x));
            g.y = __fmaf_rn(0.114f, i2.y, __fmaf_rn(0.587f, i1.y, 0.299f * g.y));
        }
        const float2 k = pk[e];
        const float y0 = k.x * g.x, y1 = two ? k.y * g.y : 0.f;
        if (!two) w1 = 0.f;
        st2(X + o, w0, w1, two);
        st2(Y + o, y0, y1, two);
        ff_add(m[0], mlo[0], w0 + w1);
        ff_add(m[1], mlo[1], __fmaf_rn(w0, w0, w1 * w1));
        ff_add(m[2], mlo[2], y0 + y1);
        ff_add(m[3], mlo[3], __fmaf_rn(y0, y0, y1 * y1));
    }
};

template <bool GRAY3>
__global__ void __launch_bounds__(32 * FS_WARPS, 4) k_final_pce(FinalArgs a) {
    __shared__ double sh[FS_WARPS][4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cg = blockIdx.x * FS_WARPS + warp;
    const int z = blockIdx.z;
    const long long hw = (long long)a.H * a.W;
    const long long A = (long long)a.Rc * a.Cc;
    const bool vec = (a.W % 2 == 0) && (((reinterpret_cast<uintptr_t>(a.Xo) | reinterpret_cast<uintptr_t>(a.Yo) |
                                          reinterpret_cast<uintptr_t>(a.Kq) | reinterpret_cast<uintptr_t>(a.Iq)) &
                                         7u) == 0) && (a.k_stride % 2 == 0);
    PceEpi epi{a.Xo + z * hw, a.Yo + z * hw, a.Kq + z * a.k_stride, a.Iq + (long long)z * a.C * hw, hw, a.W, a.C,
               vec};
    if (cg * FS_COLS < a.Cc) {  // warp-uniform
        const long long doff = (GRAY3 ? 3LL : 1LL) * z * A;
        const float *LL = a.LL ? static_cast<const float *>(a.LL) + z * A : nullptr;
        stream_synth<GRAY3, float>(LL, static_cast<const float *>(a.LH) + doff, static_cast<const float *>(a.HL) + doff,
                            static_cast<const float *>(a.HH) + doff, A, a.Rc, a.Cc, a.f, cg, blockIdx.y * FS_ROWS,
                            a.H, a.W, epi);
    }
    double v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = (double)epi.m[k] + (double)epi.mlo[k];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int w = 0; w < FS_WARPS; ++w) t += sh[w][threadIdx.x];
        const long long blk = (long long)blockIdx.y * gridDim.x + blockIdx.x;
        a.part_m[((long long)z * gridDim.x * gridDim.y + blk) * 4 + threadIdx.x] = t;
    }
}

static dim3 stream_grid(int Rc, int Cc, int planes) {
    const int groups = (Cc + FS_COLS - 1) / FS_COLS;
    return dim3((unsigned)((groups + FS_WARPS - 1) / FS_WARPS), (unsigned)((Rc + FS_ROWS - 1) / FS_ROWS),
                (unsigned)planes);
}

// The streaming form pays off when its grid fills the GPU; small planes
// (deep levels, small images) keep the tiled kernels.
static bool stream_pays(int Rc, int Cc, int planes) {
    const dim3 g = stream_grid(Rc, Cc, planes);
    return (long long)g.x * g.y * g.z * FS_WARPS >= 3648;  // half of 152 SMs x 48 warps
}

int final_pce_blocks(int Rc, int Cc) {
    const dim3 g = stream_grid(Rc, Cc, 1);
    return (int)(g.x * g.y);
}

template <class T>
static void launch_synthesis_stream(const SynArgs &a, cudaStream_t st) {
    k_synthesis_stream<false, T><<<stream_grid(a.Rc, a.Cc, a.P), 32 * FS_WARPS, 0, st>>>(a);
}

cudaError_t launch_synthesis(const SynArgs &a, cudaStream_t st, int choice) {
    const bool stream = choice == 1 || (choice == 0 && stream_pays(a.Rc, a.Cc, a.P));
    if (a.gray3) {  // float32 only (checked by the caller)
        k_synthesis_stream<true, float><<<stream_grid(a.Rc, a.Cc, a.P), 32 * FS_WARPS, 0, st>>>(a);
        return cudaGetLastError();
    }
    if (stream) {
        if (a.sdt == SB_F16)
            launch_synthesis_stream<__half>(a, st);
        else if (a.sdt == SB_BF16)
            launch_synthesis_stream<__nv_bfloat16>(a, st);
        else
            launch_synthesis_stream<float>(a, st);
        return cudaGetLastError();
    }
    dim3 block(32, 8);
    dim3 grid((unsigned)((2 * a.Cc + OT - 1) / OT), (unsigned)((2 * a.Rc + OT - 1) / OT), (unsigned)a.P);
    if (a.sdt == SB_F16)
        k_synthesis<__half><<<grid, block, 0, st>>>(a);
    else if (a.sdt == SB_BF16)
        k_synthesis<__nv_bfloat16><<<grid, block, 0, st>>>(a);
    else
        k_synthesis<float><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

template <class T>
static void launch_final_t(const FinalArgs &a, bool mle, cudaStream_t st) {
    dim3 block(32, 8);
    dim3 grid((unsigned)((a.W + OT - 1) / OT), (unsigned)((a.H + OT - 1) / OT), (unsigned)(mle ? a.C : a.C * a.G));
    if (!mle)
        k_final<false, T, false><<<grid, block, 0, st>>>(a);
    else if (a.compensated)
        k_final<true, T, true><<<grid, block, 0, st>>>(a);
    else
        k_final<true, T, false><<<grid, block, 0, st>>>(a);
}

// MLE mode, wide tile: float32 subbands (16-byte aligned, Cc a multiple of 4
// so no staged chunk straddles the periodic wrap), even W and 8-byte aligned
// group sums
constexpr int kFinalWideBuf = 2;
static bool final_wide_ok(const FinalArgs &a) {
    const uintptr_t sb = (a.LL ? reinterpret_cast<uintptr_t>(a.LL) : 0) | reinterpret_cast<uintptr_t>(a.LH) |
                         reinterpret_cast<uintptr_t>(a.HL) | reinterpret_cast<uintptr_t>(a.HH);
    return a.sdt == SB_F32 && a.Cc % 4 == 0 && a.W % 2 == 0 && (sb & 15u) == 0 &&
           (reinterpret_cast<uintptr_t>(a.X) & 7u) == 0;
}
template <bool COMP>
static void launch_final_wide(const FinalArgs &a, cudaStream_t st) {
    constexpr int BUF = kFinalWideBuf;
    const size_t smem = sizeof(AsyncTileW<BUF>);
    cudaFuncSetAttribute(k_final_async_w<COMP, BUF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const dim3 grid((unsigned)((a.W + AW_OW - 1) / AW_OW), (unsigned)((a.H + AW_OH - 1) / AW_OH), (unsigned)a.C);
    k_final_async_w<COMP, BUF><<<grid, 256, smem, st>>>(a);
}

// MLE mode: the copy-pipelined kernel for every subband type
template <class T>
static void launch_final_async_mle(const FinalArgs &a, cudaStream_t st) {
    dim3 block(32, 8);
    dim3 grid((unsigned)((a.W + OT - 1) / OT), (unsigned)((a.H + OT - 1) / OT), (unsigned)a.C);
    if (a.compensated)
        k_final_async<true, T><<<grid, block, 0, st>>>(a);
    else
        k_final_async<false, T><<<grid, block, 0, st>>>(a);
}

template <class T>
static void launch_final_stream(const FinalArgs &a, cudaStream_t st) {
    if (a.accumulate)
        k_final_stream<true, T><<<stream_grid(a.Rc, a.Cc, a.C * a.G), 32 * FS_WARPS, 0, st>>>(a);
    else
        k_final_stream<false, T><<<stream_grid(a.Rc, a.Cc, a.C * a.G), 32 * FS_WARPS, 0, st>>>(a);
}

cudaError_t launch_final(const FinalArgs &a, bool mle, cudaStream_t st, int choice) {
    if (mle && choice != 2 && final_wide_ok(a)) {
        if (a.compensated)
            launch_final_wide<true>(a, st);
        else
            launch_final_wide<false>(a, st);
        return cudaGetLastError();
    }
    if (mle) {
        if (a.sdt == SB_F16)
            launch_final_async_mle<__half>(a, st);
        else if (a.sdt == SB_BF16)
            launch_final_async_mle<__nv_bfloat16>(a, st);
        else
            launch_final_async_mle<float>(a, st);
        return cudaGetLastError();
    }
    if (a.pce) {  // float32 subbands only (checked by the caller)
        if (a.C == 3)
            k_final_pce<true><<<stream_grid(a.Rc, a.Cc, a.G), 32 * FS_WARPS, 0, st>>>(a);
        else
            k_final_pce<false><<<stream_grid(a.Rc, a.Cc, a.G), 32 * FS_WARPS, 0, st>>>(a);
        return cudaGetLastError();
    }
    if (stream_pays(a.Rc, a.Cc, a.C * a.G)) {
        if (a.sdt == SB_F16)
            launch_final_stream<__half>(a, st);
        else if (a.sdt == SB_BF16)
            launch_final_stream<__nv_bfloat16>(a, st);
        else
            launch_final_stream<float>(a, st);
        return cudaGetLastError();
    }
    if (a.sdt == SB_F16)
        launch_final_t<__half>(a, mle, st);
    else if (a.sdt == SB_BF16)
        launch_final_t<__nv_bfloat16>(a, mle, st);
    else
        launch_final_t<float>(a, mle, st);
    return cudaGetLastError();
}

}  // namespace prnu
