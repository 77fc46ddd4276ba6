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

struct SynTile {
    float c[4][CT][CT + 1];
    float lo[OT][CT + 1], hi[OT][CT + 1];
};

// Stage the four coefficient tiles of output tile (y0, x0) of one plane.
__device__ __forceinline__ void load_coeffs(SynTile &s, const float *LL, const float *LH, const float *HL,
                                            const float *HH, long long poff, int Rc, int Cc, int y0, int x0,
                                            int tid) {
    const int m0 = (y0 >> 1) - 3, n0 = (x0 >> 1) - 3;
    for (int i = tid; i < CT * CT; i += 256) {
        const int r = i / CT, c = i - r * CT;
        const long long o = poff + (long long)wrap(m0 + r, Rc) * Cc + wrap(n0 + c, Cc);
        s.c[0][r][c] = LL ? __ldg(LL + o) : 0.f;
        s.c[1][r][c] = __ldg(LH + o);
        s.c[2][r][c] = __ldg(HL + o);
        s.c[3][r][c] = __ldg(HH + o);
    }
}

// Column synthesis into lo/hi, then row synthesis of one output sample.
__device__ __forceinline__ void synth_cols(SynTile &s, const Filt &f, int tid) {
    for (int i = tid; i < OT * CT; i += 256) {
        const int y = i / CT, c = i - y * CT;
        const int e = y & 1, mr = (y >> 1) + 3;
        float lo = 0.f, hi = 0.f;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float hk = f.h[e + 2 * t], gk = f.g[e + 2 * t];
            lo = __fmaf_rn(hk, s.c[0][mr - t][c], lo);
            lo = __fmaf_rn(gk, s.c[1][mr - t][c], lo);
            hi = __fmaf_rn(hk, s.c[2][mr - t][c], hi);
            hi = __fmaf_rn(gk, s.c[3][mr - t][c], hi);
        }
        s.lo[y][c] = lo;
        s.hi[y][c] = hi;
    }
}

__device__ __forceinline__ float synth_row(const SynTile &s, const Filt &f, int y, int x) {
    const int e = x & 1, nr = (x >> 1) + 3;
    float v = 0.f;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        v = __fmaf_rn(f.h[e + 2 * t], s.lo[y][nr - t], v);
        v = __fmaf_rn(f.g[e + 2 * t], s.hi[y][nr - t], v);
    }
    return v;
}

__global__ void __launch_bounds__(256) k_synthesis(SynArgs a) {
    __shared__ SynTile s;
    const int plane = blockIdx.z;
    const int y0 = blockIdx.y * OT, x0 = blockIdx.x * OT;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const long long poff = (long long)plane * a.Rc * a.Cc;
    load_coeffs(s, a.LL, a.LH, a.HL, a.HH, poff, a.Rc, a.Cc, y0, x0, tid);
    __syncthreads();
    synth_cols(s, a.f, tid);
    __syncthreads();
    const int Ro = 2 * a.Rc, Co = 2 * a.Cc;
    const int x = threadIdx.x;
    for (int yl = threadIdx.y; yl < OT; yl += blockDim.y) {
        const int gy = y0 + yl, gx = x0 + x;
        if (gy < Ro && gx < Co) a.out[((long long)plane * Ro + gy) * Co + gx] = synth_row(s, a.f, yl, x);
    }
}

// Level 1: W for the cropped H x W region; residual or MLE accumulation.
template <bool MLE>
__global__ void __launch_bounds__(256) k_final(FinalArgs a) {
    __shared__ SynTile s;
    const int c = blockIdx.z;
    const int y0 = blockIdx.y * OT, x0 = blockIdx.x * OT;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int x = threadIdx.x;
    constexpr int PER = OT / 8;  // rows per thread
    float an[PER], ad[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) { an[k] = 0.f; ad[k] = 0.f; }
    const long long hw = (long long)a.H * a.W;
    for (int i = 0; i < a.G; ++i) {
        const int plane = i * a.C + c;
        const long long poff = (long long)plane * a.Rc * a.Cc;
        if (i > 0) __syncthreads();
        load_coeffs(s, a.LL, a.LH, a.HL, a.HH, poff, a.Rc, a.Cc, y0, x0, tid);
        __syncthreads();
        synth_cols(s, a.f, tid);
        __syncthreads();
        const float fn = MLE ? (float)a.sc.count(plane) : 1.f;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int yl = threadIdx.y + 8 * k;
            const int gy = y0 + yl, gx = x0 + x;
            if (gy < a.H && gx < a.W) {
                const float w = synth_row(s, a.f, yl, x);
                if (MLE) {
                    const float I = __fdiv_rn(__ldg(a.X + (long long)plane * hw + (long long)gy * a.W + gx), fn);
                    an[k] = __fmaf_rn(w, I, an[k]);
                    ad[k] = __fmaf_rn(I, I, ad[k]);
                } else {
                    a.res_out[(long long)c * hw + (long long)gy * a.W + gx] = w;
                }
            }
        }
    }
    if (MLE) {
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int gy = y0 + threadIdx.y + 8 * k, gx = x0 + x;
            if (gy < a.H && gx < a.W) {
                const long long o = (long long)c * hw + (long long)gy * a.W + gx;
                a.num[o] += an[k];
                a.den[o] += ad[k];
            }
        }
    }
}

cudaError_t launch_synthesis(const SynArgs &a, cudaStream_t st) {
    dim3 block(32, 8);
    dim3 grid((unsigned)((2 * a.Cc + OT - 1) / OT), (unsigned)((2 * a.Rc + OT - 1) / OT), (unsigned)a.P);
    k_synthesis<<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_final(const FinalArgs &a, bool mle, cudaStream_t st) {
    dim3 block(32, 8);
    dim3 grid((unsigned)((a.W + OT - 1) / OT), (unsigned)((a.H + OT - 1) / OT), (unsigned)a.C);
    if (mle)
        k_final<true><<<grid, block, 0, st>>>(a);
    else
        k_final<false><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace prnu
