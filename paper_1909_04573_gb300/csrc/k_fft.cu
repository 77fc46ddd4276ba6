// k_fft.cu -- once-per-fingerprint and once-per-query steps:
//   finalize: K = num/den (Sec. III-A) in float64, optional grey conversion,
//             zero-mean (column means, then row means) and DFT-domain Wiener
//             filter (literature steps the paper does not define);
//   PCE:      peak-to-correlation energy of a query (Sec. IV, threshold 60;
//             defined there by citation only).
// The DFTs go through cuFFT (float32); every sum that decides a result (means,
// variance, correlation energy) is accumulated in float64 with a fixed
// two-stage reduction, so results do not change from run to run.
#include <cufft.h>

#include <algorithm>
#include <climits>
#include <cmath>

#include "kernels.cuh"

namespace prnu {

constexpr int RB = 256;  // reduction block size

__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
    __syncthreads();
    return t;  // valid in thread 0
}

// ---------------------------------------------------------------- finalize --
// K = num/den to float64 accuracy in float32 arithmetic (GB300's float64 rate
// is a small fraction of its float32 rate): q0 = num * (1/den) is within about
// an ulp of the quotient, so r = num - q0 den is exact (one FMA), and
// q0 + r/den is carried as an unevaluated float-float pair (hi, lo), accurate
// to O(2^-44) relative; q0 need not be the correctly rounded quotient, the
// residual carries its error.
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF div_ff(float n, float d) {
    const float rd = __frcp_rn(d);
    const float q0 = __fmul_rn(n, rd);
    const float r = __fmaf_rn(-q0, d, n);
    return FF{q0, __fmul_rn(r, rd)};
}
// a * (hi, lo) + (s, t) in float-float: TwoProd by FMA, then TwoSum
__device__ __forceinline__ FF ff_fma(float a, FF x, FF acc) {
    const float p = __fmul_rn(a, x.hi);
    const float pe = __fmaf_rn(a, x.hi, -p);  // exact error of the product
    float sh, se;
    two_sum(acc.hi, p, sh, se);
    const float lo = __fadd_rn(__fadd_rn(acc.lo, se), __fmaf_rn(a, x.lo, pe));
    float h, l;
    fast_two_sum(sh, lo, h, l);
    return FF{h, l};
}

// The grey weights as float-float pairs of 0.299, 0.587, 0.114.
__constant__ float kGrayHi[3] = {0.299f, 0.587f, 0.114f};
__constant__ float kGrayLo[3] = {(float)(0.299 - (double)0.299f), (float)(0.587 - (double)0.587f),
                                 (float)(0.114 - (double)0.114f)};

// num_lo / den_lo (nullable): low parts of compensated float-float sums, so
// that the quotient is (num + num_lo) / (den + den_lo).
__global__ void k_divide(const float *num, const float *den, const float *num_lo, const float *den_lo, long long hw,
                         int C, int gray, float *K) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < hw;
         i += (long long)gridDim.x * blockDim.x) {
        // every load of the pixel first, so their latencies overlap (no load
        // waits on a value loaded before it)
        float dv[3] = {0.f, 0.f, 0.f}, nv[3] = {0.f, 0.f, 0.f}, dlv[3] = {0.f, 0.f, 0.f}, nlv[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (c < C) {
                const long long o = c * hw + i;
                dv[c] = den[o];
                nv[c] = num[o];
                if (num_lo) {
                    dlv[c] = den_lo[o];
                    nlv[c] = num_lo[o];
                }
            }
        }
        FF k[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (c >= C) break;
            const float d = dv[c];
            if (num_lo) {
                // (n + nl) / (d + dl): q0 from the high parts, then the exact residual of the pair
                const float dl = dlv[c];
                if (d == 0.f && dl == 0.f) {
                    k[c] = FF{0.f, 0.f};
                    continue;
                }
                float dh, dlo;
                fast_two_sum(d, dl, dh, dlo);
                const float n = nv[c], nl = nlv[c];
                const float q0 = __fdiv_rn(__fadd_rn(n, nl), dh);
                // r = (n + nl) - q0 (dh + dlo), accurate to the float-float level
                const float p = __fmul_rn(q0, dh), pe = __fmaf_rn(q0, dh, -p);
                const float r = __fadd_rn(__fadd_rn(__fsub_rn(n, p), nl), -__fmaf_rn(q0, dlo, pe));
                k[c] = FF{q0, __fmul_rn(r, __frcp_rn(dh))};
            } else {
                k[c] = d != 0.f ? div_ff(nv[c], d) : FF{0.f, 0.f};
            }
        }
        if (gray) {
            FF acc{0.f, 0.f};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                acc = ff_fma(kGrayHi[c], k[c], acc);
                acc = ff_fma(kGrayLo[c], FF{k[c].hi, 0.f}, acc);
            }
            K[i] = __fadd_rn(acc.hi, acc.lo);
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c)
                if (c < C) K[c * hw + i] = __fadd_rn(k[c].hi, k[c].lo);
        }
    }
}

// Float-float helpers: sums kept as (hi, lo) pairs with TwoSum (no float64
// arithmetic per element; float64 only for the few per-block partials).
__device__ __forceinline__ void ffa(FF &a, float v) { ff_add(a.hi, a.lo, v); }
__device__ __forceinline__ double ffd(const FF &a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ FF ff_of(double v) {
    const float h = (float)v;
    return FF{h, (float)(v - (double)h)};
}
// (x - m) for a float x and a float-float m, as a float-float value
__device__ __forceinline__ FF ff_sub(float x, FF m) {
    float s, e;
    two_sum(x, -m.hi, s, e);
    return FF{s, __fsub_rn(e, m.lo)};
}

// column means of one plane in two passes: a 2-D grid of partial column
// sums over row bands (coalesced across threads), then one thread per column
// sums its bands in order.
constexpr int CM_BAND = 64;
__global__ void k_colsum_part(const float *K, int H, int W, double *part) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int band = blockIdx.y;
    if (x >= W) return;
    const int y0 = band * CM_BAND, y1 = min(H, y0 + CM_BAND);
    FF s{0.f, 0.f};
#pragma unroll 8
    for (int y = y0; y < y1; ++y) ffa(s, K[(long long)y * W + x]);  // loads of 8 rows in flight
    part[(long long)band * W + x] = ffd(s);
}

// column means as float-float pairs (each in its 8-byte slot)
__global__ void k_colmean(const double *part, int H, int W, FF *colmean) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= W) return;
    const int nb = (H + CM_BAND - 1) / CM_BAND;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(long long)b * W + x];
    colmean[x] = ff_of(s / H);
}

// row means of K - colmean (float-float pairs): one block per row
__global__ void k_rowmean(const float *K, int H, int W, const FF *colmean, FF *rowmean) {
    __shared__ double sh[32];
    const int y = blockIdx.x;
    FF acc{0.f, 0.f};
#pragma unroll 4
    for (int x = threadIdx.x; x < W; x += blockDim.x) {  // four columns' loads in flight
        const FF d = ff_sub(K[(long long)y * W + x], colmean[x]);
        ffa(acc, d.hi);
        ffa(acc, d.lo);
    }
    const double s = block_sum(ffd(acc), sh);
    if (threadIdx.x == 0) rowmean[y] = ff_of(s / W);
}

// K - colmean - rowmean, rounded once; rows over blocks, columns over threads
// (the means are separate buffers, so a column's loads need not wait for the
// previous column's store)
__global__ void k_sub_means(float *__restrict__ K, int H, int W, const FF *__restrict__ colmean,
                            const FF *__restrict__ rowmean) {
    for (int y = blockIdx.x; y < H; y += gridDim.x) {
        const FF rm = rowmean[y];
        float *row = K + (long long)y * W;
#pragma unroll 4
        for (int x = threadIdx.x; x < W; x += blockDim.x) {
            const FF cm = colmean[x];
            const FF a = ff_sub(row[x], cm);  // a.hi + a.lo = K - colmean
            float s, e;
            two_sum(a.hi, -rm.hi, s, e);
            row[x] = __fadd_rn(s, __fadd_rn(__fsub_rn(e, rm.lo), a.lo));
        }
    }
}

// stage 1 of sum and sum of squares about `center` (nullable => 0)
__global__ void k_moments(const float *v, long long n, const double *center, double *part) {
    __shared__ double sh[32];
    const FF c = ff_of(center ? center[0] : 0.0);
    FF s{0.f, 0.f}, q{0.f, 0.f};
#pragma unroll 4
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {  // four loads in flight
        const FF d = ff_sub(v[i], c);
        ffa(s, d.hi);
        ffa(s, d.lo);
        // d^2 with the product error of hi^2 (TwoProd by FMA); the lo terms are far below it
        const float p = __fmul_rn(d.hi, d.hi);
        ffa(q, p);
        ffa(q, __fmaf_rn(d.hi, d.hi, -p) + 2.f * d.hi * d.lo);
    }
    const double ss = block_sum(ffd(s), sh);
    const double qq = block_sum(ffd(q), sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = ss;
        part[2 * blockIdx.x + 1] = qq;
    }
}

// stage 2: out[0] = center + mean, out[1] = sum of squares about center / n,
// less the squared mean of the deviations when `central` (one pass about 0)
__global__ void k_moments_final(const double *part, int nb, long long n, const double *center, double *out,
                                int central) {
    __shared__ double sh[32];
    double s = 0.0, q = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        s += part[2 * i];
        q += part[2 * i + 1];
    }
    s = block_sum(s, sh);
    q = block_sum(q, sh);
    if (threadIdx.x == 0) {
        const double c = center ? center[0] : 0.0;
        const double m = s / (double)n;
        out[0] = c + m;
        out[1] = central ? q / (double)n - m * m : q / (double)n;
    }
}

// DFT-domain Wiener on the half spectrum of a real plane.  |F| is point
// symmetric (F(-k) = conj F(k)) and so are the windows, so the shrunk
// magnitudes and the ratio Mn/M are too: the full magnitude plane is built
// from the half spectrum, and the ratio is applied to the half spectrum
// before a complex-to-real inverse.
__global__ void k_magnitude_half(const cufftComplex *Fh, int H, int W, float inv_sqrt_n, float *M) {
    const int W2 = W / 2 + 1;
    for (int y = blockIdx.x; y < H; y += gridDim.x) {
        const cufftComplex *row = Fh + (long long)y * W2;
        const cufftComplex *mrow = Fh + (long long)((H - y) % H) * W2;  // row of -ky
        for (int x = threadIdx.x; x < W; x += blockDim.x) {
            const cufftComplex v = x < W2 ? row[x] : mrow[W - x];
            M[(long long)y * W + x] = hypotf(v.x, v.y) * inv_sqrt_n;
        }
    }
}

// Fh *= scale * Mn/M (0 where M == 0) over the half spectrum
__global__ void k_apply_ratio_half(cufftComplex *Fh, const float *M, const float *Mn, int H, int W, float scale) {
    const int W2 = W / 2 + 1;
    for (int y = blockIdx.x; y < H; y += gridDim.x)
        for (int x = threadIdx.x; x < W2; x += blockDim.x) {
            const long long o = (long long)y * W + x;
            const float m = M[o];
            const float r = m > 0.f ? __fdiv_rn(Mn[o], m) * scale : 0.f;
            cufftComplex &f = Fh[(long long)y * W2 + x];
            f.x *= r;
            f.y *= r;
        }
}

// -------------------------------------------------------------------- PCE --
// Batched over n queries (grid y = query).  X_i = grey(residual_i),
// Y_i = K * grey(img_i); the block partials carry sum and sum of squares of
// X_i and Y_i in float64.  The means are removed exactly by zeroing the DC
// bin of the cross spectrum: sum_x (X-mx)(Y(x+s)-my) = sum_x X Y(x+s) - N mx my.
__global__ void k_pce_prep(const float *Kbase, long long k_stride, const float *Wq, const float *Iq, long long hw,
                           int C, float *X, float *Y, double *part) {
    __shared__ double sh[32];
    const int q = blockIdx.y;
    const float *K = Kbase + (long long)q * k_stride;  // one fingerprint for all queries, or one per query
    const float *w = Wq + (long long)q * C * hw;
    const float *im = Iq + (long long)q * C * hw;
    float *xo = X + (long long)q * hw;
    float *yo = Y + (long long)q * hw;
    // per-thread float-float sums (float32 partials over 4 samples), float64 only across the block
    FF sx{0.f, 0.f}, sxx{0.f, 0.f}, sy{0.f, 0.f}, syy{0.f, 0.f};
    auto one = [&](float w0, float w1, float w2, float i0, float i1, float i2, float k, float &a, float &yv) {
        float b;
        if (C == 3) {
            a = __fmaf_rn(0.114f, w2, __fmaf_rn(0.587f, w1, 0.299f * w0));
            b = __fmaf_rn(0.114f, i2, __fmaf_rn(0.587f, i1, 0.299f * i0));
        } else {
            a = w0;
            b = i0;
        }
        yv = k * b;
    };
    const bool vec = ((hw & 3) == 0) && (((reinterpret_cast<uintptr_t>(Wq) | reinterpret_cast<uintptr_t>(Iq) |
                                           reinterpret_cast<uintptr_t>(K) | reinterpret_cast<uintptr_t>(X) |
                                           reinterpret_cast<uintptr_t>(Y)) & 15u) == 0);
    if (vec) {
        const long long n4 = hw >> 2;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
             i += (long long)gridDim.x * blockDim.x) {
            const float4 k4 = __ldg(reinterpret_cast<const float4 *>(K) + i);
            const float4 w0 = __ldg(reinterpret_cast<const float4 *>(w) + i);
            const float4 i0 = __ldg(reinterpret_cast<const float4 *>(im) + i);
            float4 w1 = w0, w2 = w0, i1 = i0, i2 = i0;
            if (C == 3) {
                w1 = __ldg(reinterpret_cast<const float4 *>(w + hw) + i);
                w2 = __ldg(reinterpret_cast<const float4 *>(w + 2 * hw) + i);
                i1 = __ldg(reinterpret_cast<const float4 *>(im + hw) + i);
                i2 = __ldg(reinterpret_cast<const float4 *>(im + 2 * hw) + i);
            }
            float4 xa, ya;
            one(w0.x, w1.x, w2.x, i0.x, i1.x, i2.x, k4.x, xa.x, ya.x);
            one(w0.y, w1.y, w2.y, i0.y, i1.y, i2.y, k4.y, xa.y, ya.y);
            one(w0.z, w1.z, w2.z, i0.z, i1.z, i2.z, k4.z, xa.z, ya.z);
            one(w0.w, w1.w, w2.w, i0.w, i1.w, i2.w, k4.w, xa.w, ya.w);
            reinterpret_cast<float4 *>(xo)[i] = xa;
            reinterpret_cast<float4 *>(yo)[i] = ya;
            ffa(sx, (xa.x + xa.y) + (xa.z + xa.w));
            ffa(sxx, __fmaf_rn(xa.x, xa.x, xa.y * xa.y) + __fmaf_rn(xa.z, xa.z, xa.w * xa.w));
            ffa(sy, (ya.x + ya.y) + (ya.z + ya.w));
            ffa(syy, __fmaf_rn(ya.x, ya.x, ya.y * ya.y) + __fmaf_rn(ya.z, ya.z, ya.w * ya.w));
        }
    } else {
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < hw;
             i += (long long)gridDim.x * blockDim.x) {
            float xa, ya;
            if (C == 3)
                one(w[i], w[hw + i], w[2 * hw + i], im[i], im[hw + i], im[2 * hw + i], K[i], xa, ya);
            else
                one(w[i], 0.f, 0.f, im[i], 0.f, 0.f, K[i], xa, ya);
            xo[i] = xa;
            yo[i] = ya;
            ffa(sx, xa);
            ffa(sxx, xa * xa);
            ffa(sy, ya);
            ffa(syy, ya * ya);
        }
    }
    const double bx = block_sum(ffd(sx), sh);
    const double bxx = block_sum(ffd(sxx), sh);
    const double by = block_sum(ffd(sy), sh);
    const double byy = block_sum(ffd(syy), sh);
    if (threadIdx.x == 0) {
        double *o = part + ((long long)q * gridDim.x + blockIdx.x) * 4;
        o[0] = bx;
        o[1] = bxx;
        o[2] = by;
        o[3] = byy;
    }
}

// Z_i = conj(FX_i) * FY_i with the DC bin set to 0 (C(s) = sum_x X(x) Y(x+s));
// grid y = query
__global__ void k_cross_spectrum(const cufftComplex *FX, const cufftComplex *FY, long long nh, int n,
                                 cufftComplex *Z) {
    const long long off = (long long)blockIdx.y * nh;
    const cufftComplex *fx = FX + off, *fy = FY + off;
    cufftComplex *z = Z + off;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nh;
         i += (long long)gridDim.x * blockDim.x) {
        const cufftComplex a = fx[i], b = fy[i];
        z[i] = i == 0 ? make_cuFloatComplex(0.f, 0.f)
                      : make_cuFloatComplex(__fmaf_rn(a.x, b.x, a.y * b.y), __fmaf_rn(a.x, b.y, -a.y * b.x));
    }
}

// energy outside the neighbourhood of zero shift and argmax (first index on
// ties); one row segment per iteration so the row index is known
__global__ void k_pce_energy(const float *Cr, int H, int W, int r, double *part_e, float *part_v,
                             long long *part_i) {
    __shared__ double sh[32];
    __shared__ float sv[RB];
    __shared__ long long si[RB];
    const int q = blockIdx.y;
    const long long n = (long long)H * W;
    const float *c = Cr + (long long)q * n;
    FF acc{0.f, 0.f};  // float-float energy (no float64 per row)
    float bv = -__int_as_float(0x7f800000);
    long long bi = 0x7fffffffffffffffLL;
    const bool vec = (W % 4 == 0) && ((reinterpret_cast<uintptr_t>(c) & 15u) == 0);
    auto one = [&](float v, int y, int x, bool ynear, float &fe) {
        const bool near = ynear && min(x, W - x) <= r;
        if (!near) fe = __fmaf_rn(v, v, fe);
        if (v > bv) { bv = v; bi = (long long)y * W + x; }  // scan order is increasing per thread
    };
    // rows are distributed over blocks, columns over threads
    for (int y = blockIdx.x; y < H; y += gridDim.x) {
        const bool ynear = min(y, H - y) <= r;
        const float *row = c + (long long)y * W;
        float fe = 0.f;
        if (vec) {
            for (int x4 = threadIdx.x; x4 < W / 4; x4 += blockDim.x) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(row) + x4);
                one(v.x, y, 4 * x4, ynear, fe);
                one(v.y, y, 4 * x4 + 1, ynear, fe);
                one(v.z, y, 4 * x4 + 2, ynear, fe);
                one(v.w, y, 4 * x4 + 3, ynear, fe);
            }
        } else {
            for (int x = threadIdx.x; x < W; x += blockDim.x) one(row[x], y, x, ynear, fe);
        }
        ffa(acc, fe);
    }
    const double e = block_sum(ffd(acc), sh);
    sv[threadIdx.x] = bv;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            const float ov = sv[threadIdx.x + s];
            const long long oi = si[threadIdx.x + s];
            if (ov > sv[threadIdx.x] || (ov == sv[threadIdx.x] && oi < si[threadIdx.x])) {
                sv[threadIdx.x] = ov;
                si[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const long long o = (long long)q * gridDim.x + blockIdx.x;
        part_e[o] = e;
        part_v[o] = sv[0];
        part_i[o] = si[0];
    }
}

// one block per query; C(0, 0) of query q at c0[q * c0_stride]
__global__ void k_pce_final(const float *c0, long long c0_stride, const double *part_e, const float *part_v,
                            const long long *part_i, int nb, const double *part_m, int nbm, PceScalars *out) {
    __shared__ double sh[32];
    const int q = blockIdx.x;
    double e = 0.0, m[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nb; i += blockDim.x) e += part_e[(long long)q * nb + i];
    for (int i = threadIdx.x; i < nbm; i += blockDim.x)
        for (int k = 0; k < 4; ++k) m[k] += part_m[((long long)q * nbm + i) * 4 + k];
    e = block_sum(e, sh);
    for (int k = 0; k < 4; ++k) m[k] = block_sum(m[k], sh);
    // the peak: the largest block maximum, the smallest pixel index among
    // equal ones (a strict order on the distinct (value, index) pairs, so the
    // threads' strided scans and their merge find the same pair a scan in
    // order does)
    __shared__ float wv[32];
    __shared__ long long wi[32];
    float bv = -INFINITY;
    long long bi = LLONG_MAX;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const float v = part_v[(long long)q * nb + i];
        const long long ix = part_i[(long long)q * nb + i];
        if (v > bv || (v == bv && ix < bi)) { bv = v; bi = ix; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float v = __shfl_down_sync(0xffffffffu, bv, o);
        const long long ix = __shfl_down_sync(0xffffffffu, bi, o);
        if (v > bv || (v == bv && ix < bi)) { bv = v; bi = ix; }
    }
    if ((threadIdx.x & 31) == 0) {
        wv[threadIdx.x >> 5] = bv;
        wi[threadIdx.x >> 5] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (wv[w] > bv || (wv[w] == bv && wi[w] < bi)) { bv = wv[w]; bi = wi[w]; }
        if (bi == LLONG_MAX) bi = part_i[(long long)q * nb];  // every maximum NaN: the first block's pixel
        out[q].c0 = (double)c0[(long long)q * c0_stride];
        out[q].energy = e;
        out[q].peak_idx = bi;
        out[q].sx = m[0];
        out[q].sxx = m[1];
        out[q].sy = m[2];
        out[q].syy = m[3];
    }
}

// ------------------------------------------------------------- launchers --
static inline unsigned ew_blocks(long long n, int num_sms) {
    long long b = (n + 255) / 256;
    const long long cap = (long long)num_sms * 8;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

cudaError_t launch_divide(const float *num, const float *den, const float *num_lo, const float *den_lo, long long hw,
                          int C, int gray, float *K, int sms, cudaStream_t st) {
    k_divide<<<ew_blocks(hw, sms), 256, 0, st>>>(num, den, num_lo, den_lo, hw, C, gray, K);
    return cudaGetLastError();
}

cudaError_t launch_zero_mean(float *K, int H, int W, double *colmean, double *rowmean, double *part, int sms,
                             cudaStream_t st) {
    const int nb = (H + CM_BAND - 1) / CM_BAND;
    k_colsum_part<<<dim3((W + 127) / 128, nb), 128, 0, st>>>(K, H, W, part);
    FF *cm = reinterpret_cast<FF *>(colmean), *rm = reinterpret_cast<FF *>(rowmean);  // 8-byte slots
    k_colmean<<<(W + 255) / 256, 256, 0, st>>>(part, H, W, cm);
    k_rowmean<<<H, RB, 0, st>>>(K, H, W, cm, rm);
    k_sub_means<<<(unsigned)std::min(H, sms * 8), 256, 0, st>>>(K, H, W, cm, rm);
    return cudaGetLastError();
}

// out[0] = mean, out[1] = variance (population).  Two passes about the mean;
// one pass (sum and sum of squares about 0, less the squared mean) for a
// plane whose mean is known to be near zero (zero_mean), where nothing cancels.
cudaError_t launch_mean_var(const float *v, long long n, double *part, int nb, double *tmp, double *out,
                            cudaStream_t st, bool zero_mean) {
    k_moments<<<nb, RB, 0, st>>>(v, n, nullptr, part);
    if (zero_mean) {
        k_moments_final<<<1, RB, 0, st>>>(part, nb, n, nullptr, out, 1);
        return cudaGetLastError();
    }
    k_moments_final<<<1, RB, 0, st>>>(part, nb, n, nullptr, tmp, 0);
    k_moments<<<nb, RB, 0, st>>>(v, n, tmp, part);
    k_moments_final<<<1, RB, 0, st>>>(part, nb, n, tmp, out, 0);
    // out[0] = tmp[0] + mean of deviations (a refinement of the mean)
    return cudaGetLastError();
}

cudaError_t launch_magnitude_half(const cufftComplex *Fh, int H, int W, float inv_sqrt_n, float *M, int sms,
                                  cudaStream_t st) {
    k_magnitude_half<<<(unsigned)std::min(H, sms * 8), 256, 0, st>>>(Fh, H, W, inv_sqrt_n, M);
    return cudaGetLastError();
}
cudaError_t launch_apply_ratio_half(cufftComplex *Fh, const float *M, const float *Mn, int H, int W, float scale,
                                    int sms, cudaStream_t st) {
    k_apply_ratio_half<<<(unsigned)std::min(H, sms * 8), 256, 0, st>>>(Fh, M, Mn, H, W, scale);
    return cudaGetLastError();
}
cudaError_t launch_pce_prep(const float *K, long long k_stride, const float *Wq, const float *Iq, long long hw, int C,
                            int n, int nb, float *X, float *Y, double *part, cudaStream_t st) {
    k_pce_prep<<<dim3(nb, n), RB, 0, st>>>(K, k_stride, Wq, Iq, hw, C, X, Y, part);
    return cudaGetLastError();
}
cudaError_t launch_cross_spectrum(const cufftComplex *FX, const cufftComplex *FY, long long nh, int n,
                                  cufftComplex *Z, int sms, cudaStream_t st) {
    k_cross_spectrum<<<dim3(ew_blocks(nh, sms), n), 256, 0, st>>>(FX, FY, nh, n, Z);
    return cudaGetLastError();
}
cudaError_t launch_pce_reduce(const float *Cr, int H, int W, int r, int n, int nb, double *part_e, float *part_v,
                              long long *part_i, const double *part_m, int nbm, void *out, cudaStream_t st) {
    k_pce_energy<<<dim3(nb, n), RB, 0, st>>>(Cr, H, W, r, part_e, part_v, part_i);
    k_pce_final<<<n, RB, 0, st>>>(Cr, (long long)H * W, part_e, part_v, part_i, nb, part_m, nbm,
                                  (PceScalars *)out);
    return cudaGetLastError();
}

cudaError_t launch_pce_final(const float *c0, long long c0_stride, int n, const double *part_e, const float *part_v,
                             const long long *part_i, int nb, const double *part_m, int nbm, void *out,
                             cudaStream_t st) {
    k_pce_final<<<n, RB, 0, st>>>(c0, c0_stride, part_e, part_v, part_i, nb, part_m, nbm, (PceScalars *)out);
    return cudaGetLastError();
}

// PCE, NCC and peak of each query from its reduction scalars, on the device
// (the same formulas the host applies after a copy): c0 and energy carry the
// unnormalised inverse-FFT factors N and N^2; PCE is invariant to them, NCC
// divides them out.
__global__ void k_pce_outputs(const PceScalars *sc, int n, long long hw, int W, int nbhd, double *pce, double *ncc,
                              int *peak) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const PceScalars s = sc[q];
    const double N = (double)hw, outside = N - (double)nbhd * nbhd;
    pce[q] = s.energy > 0.0 ? (s.c0 >= 0 ? 1.0 : -1.0) * s.c0 * s.c0 * outside / s.energy : 0.0;
    if (ncc) {
        const double nx2 = s.sxx - s.sx * s.sx / N, ny2 = s.syy - s.sy * s.sy / N;
        ncc[q] = (nx2 > 0.0 && ny2 > 0.0) ? (s.c0 / N) / sqrt(nx2 * ny2) : 0.0;
    }
    if (peak) {
        peak[2 * q] = (int)(s.peak_idx / W);
        peak[2 * q + 1] = (int)(s.peak_idx % W);
    }
}

cudaError_t launch_pce_outputs(const void *sc, int n, long long hw, int W, int nbhd, double *pce, double *ncc,
                               int *peak, cudaStream_t st) {
    k_pce_outputs<<<(n + 127) / 128, 128, 0, st>>>(static_cast<const PceScalars *>(sc), n, hw, W, nbhd, pce, ncc,
                                                   peak);
    return cudaGetLastError();
}

size_t pce_scalars_bytes() { return sizeof(PceScalars); }

void pce_unpack(const void *p, int q, double *c0, double *energy, long long *peak_idx, double *sx, double *sxx,
                double *sy, double *syy) {
    const PceScalars *s = (const PceScalars *)p + q;
    *c0 = s->c0;
    *energy = s->energy;
    *peak_idx = s->peak_idx;
    *sx = s->sx;
    *sxx = s->sxx;
    *sy = s->sy;
    *syy = s->syy;
}

}  // namespace prnu
