// k_persist.cu -- the MLE fingerprint sums of many cameras (Sec. III-A over
// the SDA frames of Sec. III-B: group sums, wavelet denoiser, residual
// W = I - F(I), num += W I, den += I^2) as ONE persistent launch.
//
// Every block of the grid loops: claim the next item of a device work queue
// (one atomic on the queue head), wait until the items it depends on have
// completed, run it, count it as completed.  An item is one tile of one stage
// of one SDA group; the stages of a group and their inputs are
//   SDA sums (frames)       -> X                 row segment of 1024 / 4096 px
//   analysis of level l     -> LL_l, details_l    16 x 32 outputs of one plane
//   shrink of level l       -> noise_l            32 x 32 of one subband plane
//   synthesis of level l>=2 -> noise LL_{l-1}     32 x 32 outputs of one plane
//   level-1 synthesis + MLE -> num, den           32 x 32 outputs of one channel
// and an item depends on whole stages: analysis l on analysis l-1 (SDA sums
// at l = 1), shrink l on analysis l, synthesis l on shrink l and synthesis
// l+1, the MLE step on shrink 1, synthesis 2 and the MLE step of the camera's
// previous group (so num/den see one group at a time, in order), and the SDA
// sums of group g on the MLE step of group g - slots (whose workspace slot it
// reuses).  The host orders the queue so that every item's dependencies come
// earlier in it; since blocks claim items in queue order, every item a block
// waits for has been claimed by a running block, so the waits end.  Each wait
// is bounded all the same: after budget_ns of the global timer it records
// PRNU_ETIMEOUT and the failing item in the queue header and the block
// returns; every other block stops claiming once the status is set.
//
// The queue interleaves the stages of consecutive groups (the host's "waves":
// the SDA sums of group w beside the analysis of group w-1 and the synthesis
// of group w-2), so the frame reads, bound by HBM, run on the same SMs and at
// the same time as the denoising of earlier groups, bound by instruction issue.
//
// Intermediates are written and read inside the launch, so they are loaded
// with ld.global.cg (L2, coherent across SMs) or cp.async.cg, never through
// the non-coherent L1 path; the frames, which no item writes, use streaming
// loads.  float32 subbands and uint8 frames.
#include <cstring>

#include "kernels.cuh"

namespace prnu {

namespace {

constexpr float kSqrt2p = 1.41421356237309504880f;
constexpr int kThreads = 256;

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ float ldc(const float *p) { return __ldcg(p); }

// ---------------------------------------------------------------- SDA sums --
// Exact per-group byte sums of one row segment (as k_sda_sum: 16-byte
// streaming loads, two 16-bit lanes per 32-bit register, flushed every 256
// frames), transposed through shared memory into the planar X.
constexpr int kSdaPrefetch = 8;  // frames ahead of the group sums' loads that L2 is asked for
template <int C, int SEG>
__device__ void st_sda(const PGroup &g, int H, int W, float *X, int y, int seg, float *sbuf, int tid) {
    constexpr int NT = SEG * C / 16;
    static_assert(NT <= kThreads, "one 16-byte chunk per thread");
    const int rowbytes = W * C;
    const long long plane = (long long)H * W;
    const int x0 = seg * SEG;
    const int npx = min(SEG, W - x0);
    const int b0 = x0 * C + 16 * tid;
    const int nb = tid < NT ? min(16, rowbytes - b0) : 0;
    uint32_t tot[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) tot[i] = 0;
    if (nb > 0) {
        const uint8_t *fr = g.frames;
        const long long fs = g.frame_stride, rp = g.row_pitch;
        const uint8_t *base = fr + (long long)y * rp + b0;
        const bool al16 = ((reinterpret_cast<uintptr_t>(fr) | (uintptr_t)fs | (uintptr_t)rp) & 15u) == 0;
        if (al16 && nb == 16) {
            // thread 0 asks L2 for the row segment kSdaPrefetch frames ahead (bulk
            // prefetch, fire and forget), so the 16-byte loads find it in L2
            const uint8_t *segp = fr + (long long)y * rp + (long long)x0 * C;
            const unsigned segb = (unsigned)(min(SEG * C, rowbytes - x0 * C) & ~15);
            for (int jb = 0; jb < g.n; jb += 256) {
                const int je = min(g.n, jb + 256);
                uint32_t ev[4] = {0, 0, 0, 0}, od[4] = {0, 0, 0, 0};
                const uint8_t *p = base + (long long)jb * fs;
#pragma unroll 4
                for (int j = jb; j < je; ++j, p += fs) {
                    if (tid == 0 && j + kSdaPrefetch < g.n && segb)
                        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(
                                         segp + (long long)(j + kSdaPrefetch) * fs),
                                     "r"(segb)
                                     : "memory");
                    const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(p));
                    const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        ev[q] += w4[q] & 0x00FF00FFu;
                        od[q] += (w4[q] >> 8) & 0x00FF00FFu;
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    tot[4 * q + 0] += ev[q] & 0xFFFFu;
                    tot[4 * q + 1] += od[q] & 0xFFFFu;
                    tot[4 * q + 2] += ev[q] >> 16;
                    tot[4 * q + 3] += od[q] >> 16;
                }
            }
        } else {
            for (int j = 0; j < g.n; ++j) {
                const uint8_t *p = base + (long long)j * fs;
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (i < nb) tot[i] += p[i];
            }
        }
    }
    if (tid < NT) {
#pragma unroll
        for (int i = 0; i < 16; ++i) sbuf[16 * tid + i] = (float)tot[i];
    }
    __syncthreads();
    float *o = X + (long long)y * W + x0;
#pragma unroll
    for (int c = 0; c < C; ++c)
        for (int x = tid; x < npx; x += kThreads) o[(long long)c * plane + x] = sbuf[x * C + c];
}

// ---------------------------------------------------------------- analysis --
// One 16 x 32 output tile of one level of the periodised analysis, in the
// difference form of k_dwt.cu (row pass on differences to the first sample
// of each support, LL as a float-float pair, details scaled by 1/count).
constexpr int ATP = 16, ATQ = 32;
constexpr int AIR = 2 * ATP + 6, AIC = 2 * ATQ + 6, AICS = AIC + 2;
struct AnaSmem {
    float vh[AIR][AICS];
    float vl[AIR][AICS];
    float rh[AIR][ATQ + 1], rl[AIR][ATQ + 1], ss[AIR][ATQ + 1], tt[AIR][ATQ + 1];
};

template <bool LEVEL1>
__device__ void st_analysis(const float *inh, const float *inl, int R, int Cc, int H, int W, float *LLh,
                            float *LLl, float *LH, float *HL, float *HH, float scale, const Filt &f, int p0, int q0,
                            AnaSmem &s) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int R2 = R >> 1, C2 = Cc >> 1;
    const int srcW = LEVEL1 ? W : Cc;
    int srcx[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int gx = wrap_near(2 * q0 + tx + 32 * k, Cc);
        srcx[k] = LEVEL1 ? mirror(gx, W) : gx;
    }
    for (int r = ty; r < AIR; r += 8) {
        const int gy = wrap_near(2 * p0 + r, R);
        const int sy = LEVEL1 ? mirror(gy, H) : gy;
        const long long rowoff = (long long)sy * srcW;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int c = tx + 32 * k;
            if (c < AIC && PRNU_DCHECK(sy >= 0 && sy < (LEVEL1 ? H : R) && srcx[k] >= 0 && srcx[k] < srcW, rowoff + srcx[k])) {
                s.vh[r][c] = ldc(inh + rowoff + srcx[k]);
                if (!LEVEL1) s.vl[r][c] = ldc(inl + rowoff + srcx[k]);
            }
        }
    }
    __syncthreads();
    {
        const int q = tx;
        for (int r = ty; r < AIR; r += 8) {
            float v[8], w[8];
            const float2 *row = reinterpret_cast<const float2 *>(&s.vh[r][0]);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 t = row[q + j];
                v[2 * j] = t.x;
                v[2 * j + 1] = t.y;
            }
            if (!LEVEL1) {
                const float2 *rowl = reinterpret_cast<const float2 *>(&s.vl[r][0]);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float2 t = rowl[q + j];
                    w[2 * j] = t.x;
                    w[2 * j + 1] = t.y;
                }
            }
            float ss = 0.f, tt = 0.f;
#pragma unroll
            for (int k = 1; k < kTaps; ++k) {
                float dlt = __fsub_rn(v[k], v[0]);
                if (!LEVEL1) dlt = __fadd_rn(dlt, __fsub_rn(w[k], w[0]));
                ss = __fmaf_rn(f.h[k], dlt, ss);
                tt = __fmaf_rn(f.g[k], dlt, tt);
            }
            s.rh[r][q] = v[0];
            s.rl[r][q] = LEVEL1 ? 0.f : w[0];
            s.ss[r][q] = ss;
            s.tt[r][q] = tt;
        }
    }
    __syncthreads();
    const int q = tx;
#pragma unroll
    for (int pl = ty; pl < ATP; pl += 8) {
        const int p = p0 + pl, qq = q0 + q;
        if (p >= R2 || qq >= C2) continue;
        const int y0 = 2 * pl;
        const float r0h = s.rh[y0][q], r0l = s.rl[y0][q];
        float A = 0.f, B = 0.f;
#pragma unroll
        for (int j = 1; j < kTaps; ++j) {
            float D = __fsub_rn(s.rh[y0 + j][q], r0h);
            if (!LEVEL1) D = __fadd_rn(D, __fsub_rn(s.rl[y0 + j][q], r0l));
            A = __fmaf_rn(f.h[j], D, A);
            B = __fmaf_rn(f.g[j], D, B);
        }
        float Sh = 0.f, Sg = 0.f, Th = 0.f, Tg = 0.f;
#pragma unroll
        for (int j = 0; j < kTaps; ++j) {
            const float sv = s.ss[y0 + j][q], tv = s.tt[y0 + j][q];
            Sh = __fmaf_rn(f.h[j], sv, Sh);
            Sg = __fmaf_rn(f.g[j], sv, Sg);
            Th = __fmaf_rn(f.h[j], tv, Th);
            Tg = __fmaf_rn(f.g[j], tv, Tg);
        }
        const float llsmall = __fmaf_rn(kSqrt2p, A, Sh);
        const float lh = __fmaf_rn(kSqrt2p, B, Sg);
        const long long o = (long long)p * C2 + qq;
        if (LLh) {
            float sh, se, lo;
            two_sum(2.f * r0h, llsmall, sh, se);
            lo = __fadd_rn(2.f * r0l, se);
            float hh, ll;
            fast_two_sum(sh, lo, hh, ll);
            LLh[o] = hh;
            LLl[o] = ll;
        }
        LH[o] = lh * scale;
        HL[o] = Th * scale;
        HH[o] = Tg * scale;
    }
}

// ------------------------------------------------------------------ shrink --
// One 32 x 32 tile of the local-variance Wiener shrink (as k_shrink): c^2
// with a periodic halo of 4, row sums then column sums per window, minimum
// of the window means, noise coefficient c s0^2 / (max(0, m - s0^2) + s0^2).
constexpr int PST = 32, PSH = kMaxRadius, PSE = PST + 2 * PSH, PC2S = PSE + 4;
struct ShrSmem {
    float c2[PSE][PC2S];
    float rs[4][PSE][PST + 1];
};

template <bool STD>
__device__ void st_shrink(const float *in, float *out, int R, int Cc, int y0, int x0, float s2, const Win &win,
                          ShrSmem &s, int tid) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    int srcx[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) srcx[k] = wrap_near(x0 + tx + 32 * k - PSH, Cc);
    for (int r = ty; r < PSE; r += 8) {
        const long long rowoff = (long long)wrap_near(y0 + r - PSH, R) * Cc;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int c = tx + 32 * k;
            if (c < PSE) {
                const float v = ldc(in + rowoff + srcx[k]);
                s.c2[r][c] = v * v;
            }
        }
    }
    __syncthreads();
    if (STD) {
        for (int it = tid; it < PSE * (PST / 4); it += kThreads) {
            const int r = it >> 3, g = it & 7;
            const float4 *row = reinterpret_cast<const float4 *>(&s.c2[r][0]);
            float v[12];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float4 t = row[g + k];
                v[4 * k] = t.x;
                v[4 * k + 1] = t.y;
                v[4 * k + 2] = t.z;
                v[4 * k + 3] = t.w;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float a = v[j + 4];
#pragma unroll
                for (int d = 1; d <= 4; ++d) {
                    a += v[j + 4 - d] + v[j + 4 + d];
                    s.rs[d - 1][r][4 * g + j] = a;
                }
            }
        }
    } else {
        for (int r = ty; r < PSE; r += 8) {
            const int x = tx + PSH;
            for (int w = 0; w < win.n; ++w) {
                const int rad = win.r[w];
                float a = 0.f;
                for (int dx = -rad; dx <= rad; ++dx) a += s.c2[r][x + dx];
                s.rs[w][r][tx] = a;
            }
        }
    }
    __syncthreads();
    const int gx = x0 + tx;
    if (STD) {
        const int yb = 4 * ty;
        float m[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) m[k] = __int_as_float(0x7f800000);
#pragma unroll
        for (int d = 1; d <= 4; ++d) {
            float col[12];
#pragma unroll
            for (int k = 0; k < 4 + 2 * d; ++k) col[k] = s.rs[d - 1][yb + PSH - d + k][tx];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float a = 0.f;
#pragma unroll
                for (int j = 0; j <= 2 * d; ++j) a += col[k + j];
                m[k] = fminf(m[k], a * win.inv[d - 1]);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int gy = y0 + yb + k;
            if (gy >= R || gx >= Cc) continue;
            const float c = ldc(in + (long long)gy * Cc + gx);
            const float var = fmaxf(0.f, m[k] - s2);
            const float den = var + s2;
            out[(long long)gy * Cc + gx] = den > 0.f ? __fdividef(c * s2, den) : 0.f;
        }
    } else {
        for (int yl = ty; yl < PST; yl += 8) {
            const int gy = y0 + yl;
            if (gy >= R || gx >= Cc) continue;
            const int yc = yl + PSH;
            float vmin = __int_as_float(0x7f800000);
            for (int w = 0; w < win.n; ++w) {
                const int rad = win.r[w];
                float a = 0.f;
                for (int dy = -rad; dy <= rad; ++dy) a += s.rs[w][yc + dy][tx];
                vmin = fminf(vmin, a * win.inv[w]);
            }
            const float c = ldc(in + (long long)gy * Cc + gx);
            const float var = fmaxf(0.f, vmin - s2);
            const float den = var + s2;
            out[(long long)gy * Cc + gx] = den > 0.f ? __fdividef(c * s2, den) : 0.f;
        }
    }
}

// --------------------------------------------------------------- synthesis --
// One 32 x 32 output tile of the inverse DWT (gather form, columns first):
// a 19 x 19 tile (3-coefficient halo) of each of the four subbands.
constexpr int POT = 32, PCT = POT / 2 + 3, PNP = POT / 2;
struct SynSmem {
    float c[4][PCT][PCT + 1];
    float lo[POT][PCT + 1], hi[POT][PCT + 1];
};

__device__ void st_synth_cols(const float *LL, const float *LH, const float *HL, const float *HH, int Rc, int Cc,
                              int y0, int x0, const Filt &f, SynSmem &s, int tid) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    if (tx < PCT) {
        const int sx = wrap_near((x0 >> 1) - 3 + tx, Cc);
        for (int r = ty; r < PCT; r += 8) {
            const long long o = (long long)wrap_near((y0 >> 1) - 3 + r, Rc) * Cc + sx;
            s.c[0][r][tx] = LL ? ldc(LL + o) : 0.f;
            s.c[1][r][tx] = ldc(LH + o);
            s.c[2][r][tx] = ldc(HL + o);
            s.c[3][r][tx] = ldc(HH + o);
        }
    }
    __syncthreads();
    for (int it = tid; it < PNP * PCT; it += kThreads) {
        const int m = it / PCT, c = it - m * PCT;
        float a[4], b[4], u[4], v[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            a[t] = s.c[0][m + 3 - t][c];
            b[t] = s.c[1][m + 3 - t][c];
            u[t] = s.c[2][m + 3 - t][c];
            v[t] = s.c[3][m + 3 - t][c];
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            float lo = 0.f, hi = 0.f;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const float hk = f.h[e + 2 * t], gk = f.g[e + 2 * t];
                lo = __fmaf_rn(hk, a[t], lo);
                lo = __fmaf_rn(gk, b[t], lo);
                hi = __fmaf_rn(hk, u[t], hi);
                hi = __fmaf_rn(gk, v[t], hi);
            }
            s.lo[2 * m + e][c] = lo;
            s.hi[2 * m + e][c] = hi;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ float2 st_synth_pair(const SynSmem &s, const Filt &f, int y, int n) {
    float l[4], h[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        l[t] = s.lo[y][n + 3 - t];
        h[t] = s.hi[y][n + 3 - t];
    }
    float o[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        float v = 0.f;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            v = __fmaf_rn(f.h[e + 2 * t], l[t], v);
            v = __fmaf_rn(f.g[e + 2 * t], h[t], v);
        }
        o[e] = v;
    }
    return make_float2(o[0], o[1]);
}

__device__ void st_synthesis(const float *LL, const float *LH, const float *HL, const float *HH, int Rc, int Cc,
                             float *out, int y0, int x0, const Filt &f, SynSmem &s, int tid) {
    st_synth_cols(LL, LH, HL, HH, Rc, Cc, y0, x0, f, s, tid);
    const int Ro = 2 * Rc, Co = 2 * Cc;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int it = tid + kThreads * k;
        const int y = it >> 4, n = it & 15;
        const int gy = y0 + y, gx = x0 + 2 * n;
        if (gy < Ro && gx < Co) {
            const float2 v = st_synth_pair(s, f, y, n);
            float *o = out + (long long)gy * Co + gx;
            o[0] = v.x;
            o[1] = v.y;
        }
    }
}

// Level-1 synthesis of one 32 x 32 tile of one channel, cropped to H x W,
// and the MLE sums of that tile: num += W I, den += I^2 with I = X / count.
template <bool COMP>
__device__ void st_final(const float *LL, const float *LH, const float *HL, const float *HH, int Rc, int Cc,
                         const float *X, int H, int W, float inv_n, float *num, float *den, long long lo_off,
                         int y0, int x0, const Filt &f, SynSmem &s, int tid) {
    st_synth_cols(LL, LH, HL, HH, Rc, Cc, y0, x0, f, s, tid);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int it = tid + kThreads * k;
        const int y = it >> 4, n = it & 15;
        const int gy = y0 + y, gx = x0 + 2 * n;
        if (gy >= H || gx >= W) continue;
        const float2 w = st_synth_pair(s, f, y, n);
        const long long o = (long long)gy * W + gx;
        const int cnt = gx + 1 < W ? 2 : 1;
        for (int e = 0; e < cnt; ++e) {
            const float I = ldc(X + o + e) * inv_n;
            const float we = e ? w.y : w.x;
            if (COMP) {
                float h = ldc(num + o + e), l = ldc(num + lo_off + o + e);
                ff_add(h, l, we * I);
                num[o + e] = h;
                num[lo_off + o + e] = l;
                h = ldc(den + o + e);
                l = ldc(den + lo_off + o + e);
                ff_add(h, l, I * I);
                den[o + e] = h;
                den[lo_off + o + e] = l;
            } else {
                num[o + e] = __fmaf_rn(we, I, ldc(num + o + e));
                den[o + e] = __fmaf_rn(I, I, ldc(den + o + e));
            }
        }
    }
}

union PSmem {
    AnaSmem ana;
    ShrSmem shr;
    SynSmem syn;
    float sda[4096];
};

// -------------------------------------------------------------- scheduling --
struct Dep {
    int group, stage, target;
};

// The stages item (g, s) waits for (every item of each); returns how many
// (at most three).  Unused entries are set to a count that is always reached.
__device__ __forceinline__ int deps_of(const PArgs &a, int g, int s, Dep &d0, Dep &d1, Dep &d2) {
    const int L = a.L;
    auto full = [&](int dg, int ds) { return Dep{dg, ds, a.geos[a.groups[dg].geo].cnt[ds]}; };
    d0 = d1 = d2 = Dep{g, 0, 0};
    if (s == kPProbeStage) {  // diagnostic: a count nothing reaches
        d0 = Dep{g, 0, 0x7fffffff};
        return 1;
    }
    if (s == 0) {
        if (g < a.nslots) return 0;
        d0 = full(g - a.nslots, 3 * L);
        return 1;
    }
    if (s <= L) {
        d0 = full(g, s - 1);
        return 1;
    }
    if (s <= 2 * L) {
        d0 = full(g, s - L);
        return 1;
    }
    if (s < 3 * L) {
        const int l = 3 * L + 1 - s;
        d0 = full(g, L + l);
        if (l < L) {
            d1 = full(g, s - 1);
            return 2;
        }
        return 1;
    }
    d0 = full(g, L + 1);
    int n = 1;
    if (L >= 2) {
        d1 = full(g, 3 * L - 1);
        n = 2;
    }
    if (a.groups[g].prev >= 0) {
        if (n == 1)
            d1 = full(a.groups[g].prev, 3 * L);
        else
            d2 = full(a.groups[g].prev, 3 * L);
        ++n;
    }
    return n;
}

// Thread 0 of a block: wait until the completion count of d reaches its
// target (acquire), giving up after budget_ns; returns false when the launch
// has failed (here or in another block).
__device__ bool wait_dep(const PArgs &a, const Dep &d, int item, int g, int s) {
    const int *cnt = a.done + (long long)d.group * a.NS + d.stage;
    if (ld_acquire(cnt) >= d.target) return true;
    const unsigned long long t0 = gtimer();
    for (;;) {
        __nanosleep(200);
        if (ld_acquire(cnt) >= d.target) return true;
        if (ld_relaxed(&a.hdr->status) != 0) return false;
        if (gtimer() - t0 > (unsigned long long)a.budget_ns) {
            if (atomicCAS(&a.hdr->status, 0, (int)PRNU_ETIMEOUT) == 0) {
                a.hdr->fail_item = item;
                a.hdr->fail_group = g;
                a.hdr->fail_stage = s;
            }
            atomicAdd(&a.hdr->fail_blocks, 1);
            return false;
        }
    }
}

__device__ __forceinline__ bool same_or_weaker(const Dep &d, const Dep &seen) {
    return d.group == seen.group && d.stage == seen.stage && d.target <= seen.target;
}

// One queue item: tiles t*k .. t*k + k - 1 (those that exist) of stage s of
// group g, with k the stage's tiles per item.
template <bool COMP, bool STD>
__device__ void run_item(const PArgs &a, int g, int s, int t, PSmem &sm, int tid) {
    const PGroup &grp = a.groups[g];
    const PGeo &ge = a.geos[grp.geo];
    const int L = a.L, C = ge.C, H = ge.H, W = ge.W, Hp = ge.Hp, Wp = ge.Wp;
    char *slot = a.slots + (long long)(g % a.nslots) * a.slot_bytes;
    auto F = [&](long long off) { return reinterpret_cast<float *>(slot + off); };
    const float scale = __frcp_rn((float)grp.n);
    if (s == 0) {
        const int nseg = C == 3 ? (W + 1023) / 1024 : (W + 4095) / 4096;
        const int n = H * nseg;
        for (int u = t * kPTilesSda; u < min(n, (t + 1) * kPTilesSda); ++u) {
            if (u != t * kPTilesSda) __syncthreads();
            if (C == 3)
                st_sda<3, 1024>(grp, H, W, F(ge.X), u / nseg, u % nseg, sm.sda, tid);
            else
                st_sda<1, 4096>(grp, H, W, F(ge.X), u / nseg, u % nseg, sm.sda, tid);
        }
    } else if (s <= L) {
        const int l = s;
        const int R = Hp >> (l - 1), Cc = Wp >> (l - 1);
        const int R2 = R >> 1, C2 = Cc >> 1;
        const int tq = (C2 + ATQ - 1) / ATQ, tp = (R2 + ATP - 1) / ATP;
        const int n = C * tp * tq;
        const long long A = (long long)R2 * C2;
        for (int u = t * kPTilesAna; u < min(n, (t + 1) * kPTilesAna); ++u) {
            if (u != t * kPTilesAna) __syncthreads();
            const int plane = u / (tp * tq), r = u % (tp * tq);
            if (!PRNU_DCHECK(plane < C, u)) continue;
            const int p0 = (r / tq) * ATP, q0 = (r % tq) * ATQ;
            float *LLh = l < L ? F(ge.LLh[l]) + plane * A : nullptr;
            float *LLl = l < L ? F(ge.LLl[l]) + plane * A : nullptr;
            float *D = F(ge.D[l]);
            float *LH = D + plane * A, *HL = D + (C + plane) * A, *HH = D + (2 * C + plane) * A;
            if (l == 1)
                st_analysis<true>(F(ge.X) + (long long)plane * H * W, nullptr, R, Cc, H, W, LLh, LLl, LH, HL, HH,
                                  scale, a.f, p0, q0, sm.ana);
            else
                st_analysis<false>(F(ge.LLh[l - 1]) + plane * (long long)R * Cc,
                                   F(ge.LLl[l - 1]) + plane * (long long)R * Cc, R, Cc, H, W, LLh, LLl, LH, HL, HH,
                                   scale, a.f, p0, q0, sm.ana);
        }
    } else if (s <= 2 * L) {
        const int l = s - L;
        const int R = Hp >> l, Cc = Wp >> l;
        const int tq = (Cc + PST - 1) / PST, tp = (R + PST - 1) / PST;
        const int n = 3 * C * tp * tq;
        const long long A = (long long)R * Cc;
        for (int u = t * kPTilesShr; u < min(n, (t + 1) * kPTilesShr); ++u) {
            if (u != t * kPTilesShr) __syncthreads();
            const int plane = u / (tp * tq), r = u % (tp * tq);
            if (!PRNU_DCHECK(plane < 3 * C, u)) continue;
            st_shrink<STD>(F(ge.D[l]) + plane * A, F(ge.N[l]) + plane * A, R, Cc, (r / tq) * PST, (r % tq) * PST,
                           a.s2, a.win, sm.shr, tid);
        }
    } else if (s < 3 * L) {
        const int l = 3 * L + 1 - s;
        const int Rc = Hp >> l, Cc = Wp >> l;
        const int Ro = 2 * Rc, Co = 2 * Cc;
        const int tq = (Co + POT - 1) / POT, tp = (Ro + POT - 1) / POT;
        const int n = C * tp * tq;
        const long long A = (long long)Rc * Cc;
        const float *N = F(ge.N[l]);
        for (int u = t * kPTilesSyn; u < min(n, (t + 1) * kPTilesSyn); ++u) {
            if (u != t * kPTilesSyn) __syncthreads();
            const int plane = u / (tp * tq), r = u % (tp * tq);
            st_synthesis(l < L ? F(ge.Rn[l]) + plane * A : nullptr, N + plane * A, N + (C + plane) * A,
                         N + (2 * C + plane) * A, Rc, Cc, F(ge.Rn[l - 1]) + plane * (long long)Ro * Co,
                         (r / tq) * POT, (r % tq) * POT, a.f, sm.syn, tid);
        }
    } else {
        const int Rc = Hp >> 1, Cc = Wp >> 1;
        const int tq = (W + POT - 1) / POT, tp = (H + POT - 1) / POT;
        const int n = C * tp * tq;
        const long long A = (long long)Rc * Cc, hw = (long long)H * W;
        const float *N = F(ge.N[1]);
        const PCam &cam = a.cams[grp.cam];
        for (int u = t * kPTilesFin; u < min(n, (t + 1) * kPTilesFin); ++u) {
            if (u != t * kPTilesFin) __syncthreads();
            const int c = u / (tp * tq), r = u % (tp * tq);
            if (!PRNU_DCHECK(c < C, u)) continue;
            st_final<COMP>(L >= 2 ? F(ge.Rn[1]) + c * A : nullptr, N + c * A, N + (C + c) * A, N + (2 * C + c) * A,
                           Rc, Cc, F(ge.X) + c * hw, H, W, scale, cam.num + c * hw, cam.den + c * hw,
                           (long long)C * hw, (r / tq) * POT, (r % tq) * POT, a.f, sm.syn, tid);
        }
    }
}

// Thread 0: the queue item index after `it` for this block (an atomic claim),
// or -1 when the queue is empty or the launch has failed.
__device__ __forceinline__ int claim(const PArgs &a) {
    if (ld_relaxed(&a.hdr->status) != 0) return -1;
    const int it = atomicAdd(&a.hdr->next, 1);
    return it < a.total ? it : -1;
}

// Thread 0: the segment holding item `it`, walking forward from `seg`
// (claims grow with time) or bisecting when the queue has moved far ahead.
__device__ __forceinline__ int segment_of(const PArgs &a, int it, int seg) {
    if (__ldg(&a.segs[seg].start) > it) seg = 0;
    int steps = 0;
    while (seg + 1 < a.nseg && __ldg(&a.segs[seg + 1].start) <= it && steps < 8) {
        ++seg;
        ++steps;
    }
    if (seg + 1 < a.nseg && __ldg(&a.segs[seg + 1].start) <= it) {
        int lo = seg + 1, hi = a.nseg - 1;  // largest index with start <= it
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&a.segs[mid].start) <= it)
                lo = mid;
            else
                hi = mid - 1;
        }
        seg = lo;
    }
    return seg;
}

template <bool COMP, bool STD>
__global__ void __launch_bounds__(kThreads, 3) k_persist(PArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PSmem &sm = *reinterpret_cast<PSmem *>(smem_raw);
    __shared__ int s_item, s_seg, s_ok;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    // thread 0: the segment of the last item, the item claimed ahead (so the
    // claim's latency overlaps the current item), and the dependencies last
    // found complete (counts only grow, so they stay complete)
    int seg = 0, ahead = -2;
    Dep seen0{-1, 0, 0}, seen1{-1, 0, 0}, seen2{-1, 0, 0};
    for (;;) {
        if (tid == 0) {
            const int it = ahead == -2 ? claim(a) : ahead;
            if (it >= 0) seg = segment_of(a, it, seg);
            s_item = it;
            s_seg = seg;
        }
        __syncthreads();
        const int it = s_item;
        if (it < 0) break;
        const PSeg sg = a.segs[s_seg];
        if (tid == 0) {
            Dep d0, d1, d2;
            const int n = deps_of(a, sg.group, sg.stage, d0, d1, d2);
            bool ok = true;
            // entries past n are {g, 0, 0}: always complete
            if (!same_or_weaker(d0, seen0)) {
                ok = wait_dep(a, d0, it, sg.group, sg.stage);
                if (ok) seen0 = d0;
            }
            if (ok && n > 1 && !same_or_weaker(d1, seen1)) {
                ok = wait_dep(a, d1, it, sg.group, sg.stage);
                if (ok) seen1 = d1;
            }
            if (ok && n > 2 && !same_or_weaker(d2, seen2)) {
                ok = wait_dep(a, d2, it, sg.group, sg.stage);
                if (ok) seen2 = d2;
            }
            // claim the next item before running this one (deadlock-free: a
            // block's held item is always later in the queue than its running one)
            ahead = ok ? claim(a) : -1;
            s_ok = ok ? 1 : 0;
        }
        __syncthreads();
        if (!s_ok) break;
        if (sg.stage != kPProbeStage) run_item<COMP, STD>(a, sg.group, sg.stage, sg.first + (it - sg.start), sm, tid);
        __syncthreads();  // every thread's writes of the item precede its count
        if (tid == 0) {
            __threadfence();
            atomicAdd(a.done + (long long)sg.group * a.NS + sg.stage, 1);
        }
    }
}

// by-value copy of up to kPutChunk bytes into device memory (capturable)
struct PutChunk {
    unsigned int w[kPutChunk / 4];
};
__global__ void k_put_bytes(PutChunk c, int nwords, unsigned int *dst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nwords; i += gridDim.x * blockDim.x) dst[i] = c.w[i];
}

template <bool COMP, bool STD>
cudaError_t launch_persist_t(const PArgs &a, int blocks, cudaStream_t st) {
    const size_t smem = sizeof(PSmem);
    k_persist<COMP, STD><<<blocks, dim3(32, 8), smem, st>>>(a);
    return cudaGetLastError();
}

template <bool COMP, bool STD>
int blocks_per_sm_t() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_persist<COMP, STD>, kThreads, sizeof(PSmem)) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

}  // namespace

cudaError_t launch_persist(const PArgs &a, bool comp, bool std_win, int blocks, cudaStream_t st) {
    if (comp)
        return std_win ? launch_persist_t<true, true>(a, blocks, st) : launch_persist_t<true, false>(a, blocks, st);
    return std_win ? launch_persist_t<false, true>(a, blocks, st) : launch_persist_t<false, false>(a, blocks, st);
}

int persist_blocks_per_sm(bool comp, bool std_win) {
    if (comp) return std_win ? blocks_per_sm_t<true, true>() : blocks_per_sm_t<true, false>();
    return std_win ? blocks_per_sm_t<false, true>() : blocks_per_sm_t<false, false>();
}

cudaError_t launch_put_bytes(const void *src, size_t n, void *dst, cudaStream_t st) {
    const unsigned char *s = static_cast<const unsigned char *>(src);
    unsigned char *d = static_cast<unsigned char *>(dst);
    for (size_t off = 0; off < n; off += kPutChunk) {
        const size_t len = n - off < (size_t)kPutChunk ? n - off : (size_t)kPutChunk;
        PutChunk c;
        std::memset(&c, 0, sizeof c);
        std::memcpy(&c, s + off, len);
        const int nw = (int)((len + 3) / 4);
        k_put_bytes<<<(nw + 255) / 256, 256, 0, st>>>(c, nw, reinterpret_cast<unsigned int *>(d + off));
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace prnu
