// k_idwt.cu -- inverse DWT of the noise coefficients (synthesis, the
// transpose of the periodised analysis) and the fused level-1 step that forms
// the residual W = I - F(I) = IDWT(0, noise details) (Sec. III-A), crops the
// padding and either stores W or accumulates the MLE sums
// num += W I, den += I^2 (Sec. IV-A / IV-B).
//
// Gather form of x[(2n+k) mod N] += h[k] a[n] + g[k] b[n]: output sample
// j = 2m + e (e in {0, 1}) takes k = e + 2t, n = m - t for t = 0..3.
// Columns are synthesised first, then rows.  A 32 x 32 output tile needs a
// 19 x 19 tile (3-coefficient halo) of each of the four subbands.
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
    if (tx < CT) {
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
}

// Row synthesis of the output pair (y, 2n), (y, 2n+1).
__device__ __forceinline__ float2 synth_pair(const SynTile &s, const Filt &f, int y, int n) {
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
        const int cnt = gx + 1 < a.W ? 2 : 1;
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
    int cam = (MLE && a.gd) ? a.gd[0].cam : -1;  // multi-camera pass: current camera
    for (int i = 0; i < nimg; ++i) {
        const int plane = MLE ? i * a.C + (int)blockIdx.z : (int)blockIdx.z;
        if (MLE && a.gd && a.gd[i].cam != cam) {  // block-uniform: the camera changes
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
        const float inv_n = MLE ? __frcp_rn((float)a.sc.count(plane)) : 1.f;
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

cudaError_t launch_synthesis(const SynArgs &a, cudaStream_t st) {
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

cudaError_t launch_final(const FinalArgs &a, bool mle, cudaStream_t st) {
    if (a.sdt == SB_F16)
        launch_final_t<__half>(a, mle, st);
    else if (a.sdt == SB_BF16)
        launch_final_t<__nv_bfloat16>(a, mle, st);
    else
        launch_final_t<float>(a, mle, st);
    return cudaGetLastError();
}

}  // namespace prnu
