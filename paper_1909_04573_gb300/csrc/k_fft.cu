// k_fft.cu -- once-per-fingerprint and once-per-query steps:
//   finalize: K = num/den (Sec. IV-A) in float64, optional grey conversion,
//             zero-mean (column means, then row means) and DFT-domain Wiener
//             filter (literature steps the paper does not define);
//   PCE:      peak-to-correlation energy of a query (Sec. V, threshold 60;
//             defined there by citation only).
// The DFTs go through cuFFT (float32); every sum that decides a result (means,
// variance, correlation energy) is accumulated in float64 with a fixed
// two-stage reduction, so results do not change from run to run.
#include <cufft.h>

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
__global__ void k_divide(const float *num, const float *den, long long hw, int C, int gray, float *K) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < hw;
         i += (long long)gridDim.x * blockDim.x) {
        double k[3];
        for (int c = 0; c < C; ++c) {
            const double d = (double)den[c * hw + i];
            k[c] = d != 0.0 ? (double)num[c * hw + i] / d : 0.0;
        }
        if (gray) {
            K[i] = (float)(0.299 * k[0] + 0.587 * k[1] + 0.114 * k[2]);
        } else {
            for (int c = 0; c < C; ++c) K[c * hw + i] = (float)k[c];
        }
    }
}

// column means of one plane: one thread per column (coalesced across threads)
__global__ void k_colmean(const float *K, int H, int W, double *colmean) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= W) return;
    double s = 0.0;
    for (int y = 0; y < H; ++y) s += (double)K[(long long)y * W + x];
    colmean[x] = s / H;
}

// row means of K - colmean: one block per row
__global__ void k_rowmean(const float *K, int H, int W, const double *colmean, double *rowmean) {
    __shared__ double sh[32];
    const int y = blockIdx.x;
    double s = 0.0;
    for (int x = threadIdx.x; x < W; x += blockDim.x) s += (double)K[(long long)y * W + x] - colmean[x];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) rowmean[y] = s / W;
}

__global__ void k_sub_means(float *K, int H, int W, const double *colmean, const double *rowmean) {
    const long long hw = (long long)H * W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < hw;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), x = (int)(i - (long long)y * W);
        K[i] = (float)((double)K[i] - colmean[x] - rowmean[y]);
    }
}

// stage 1 of sum and sum of squares about `center` (nullable => 0)
__global__ void k_moments(const float *v, long long n, const double *center, double *part) {
    __shared__ double sh[32];
    const double c = center ? center[0] : 0.0;
    double s = 0.0, q = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double d = (double)v[i] - c;
        s += d;
        q += d * d;
    }
    s = block_sum(s, sh);
    q = block_sum(q, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s;
        part[2 * blockIdx.x + 1] = q;
    }
}

// stage 2: out[0] = center + mean, out[1] = sum of squares about center / n
__global__ void k_moments_final(const double *part, int nb, long long n, const double *center, double *out) {
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
        out[0] = c + s / (double)n;
        out[1] = q / (double)n;
    }
}

__global__ void k_to_complex(const float *K, long long n, cufftComplex *F) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        F[i] = make_cuFloatComplex(K[i], 0.f);
}

__global__ void k_magnitude(const cufftComplex *F, long long n, float inv_sqrt_n, float *M) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        M[i] = hypotf(F[i].x, F[i].y) * inv_sqrt_n;
}

// F *= Mn/M (0 where M == 0)
__global__ void k_apply_ratio(cufftComplex *F, const float *M, const float *Mn, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float m = M[i];
        const float r = m > 0.f ? __fdiv_rn(Mn[i], m) : 0.f;
        F[i].x *= r;
        F[i].y *= r;
    }
}

__global__ void k_real_scaled(const cufftComplex *F, long long n, float scale, float *K) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        K[i] = F[i].x * scale;
}

// -------------------------------------------------------------------- PCE --
// X = grey(residual_q), Y = K * grey(img_q)
__global__ void k_pce_prep(const float *K, const float *Wq, const float *Iq, long long hw, int C, float *X,
                           float *Y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < hw;
         i += (long long)gridDim.x * blockDim.x) {
        float w, im;
        if (C == 3) {
            w = (float)(0.299 * Wq[i] + 0.587 * Wq[hw + i] + 0.114 * Wq[2 * hw + i]);
            im = (float)(0.299 * Iq[i] + 0.587 * Iq[hw + i] + 0.114 * Iq[2 * hw + i]);
        } else {
            w = Wq[i];
            im = Iq[i];
        }
        X[i] = w;
        Y[i] = K[i] * im;
    }
}

__global__ void k_sub_center(float *v, long long n, const double *mean) {
    const double m = mean[0];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        v[i] = (float)((double)v[i] - m);
}

// Z = conj(FX) * FY  (C(s) = sum_x X(x) Y(x+s))
__global__ void k_cross_spectrum(const cufftComplex *FX, const cufftComplex *FY, long long n, cufftComplex *Z) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const cufftComplex a = FX[i], b = FY[i];
        Z[i] = make_cuFloatComplex(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
    }
}

struct PceScalars {
    double c0, energy, peak_val;
    long long peak_idx;
    double nx2, ny2;
};

// stage 1: energy outside the neighbourhood and argmax (first index on ties)
__global__ void k_pce_energy(const float *Cr, int H, int W, int r, double *part_e, float *part_v,
                             long long *part_i) {
    __shared__ double sh[32];
    __shared__ float sv[RB];
    __shared__ long long si[RB];
    const long long n = (long long)H * W;
    double e = 0.0;
    float bv = -__int_as_float(0x7f800000);
    long long bi = 0x7fffffffffffffffLL;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), x = (int)(i - (long long)y * W);
        const float v = Cr[i];
        const int dy = min(y, H - y), dx = min(x, W - x);  // wrapped distance to zero shift
        if (dy > r || dx > r) e += (double)v * (double)v;
        if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
    }
    e = block_sum(e, sh);
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
        part_e[blockIdx.x] = e;
        part_v[blockIdx.x] = sv[0];
        part_i[blockIdx.x] = si[0];
    }
}

__global__ void k_pce_final(const float *Cr, const double *part_e, const float *part_v, const long long *part_i,
                            int nb, const double *momx, const double *momy, PceScalars *out) {
    __shared__ double sh[32];
    double e = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) e += part_e[i];
    e = block_sum(e, sh);
    if (threadIdx.x == 0) {
        float bv = part_v[0];
        long long bi = part_i[0];
        for (int i = 1; i < nb; ++i)
            if (part_v[i] > bv || (part_v[i] == bv && part_i[i] < bi)) { bv = part_v[i]; bi = part_i[i]; }
        out->c0 = (double)Cr[0];
        out->energy = e;
        out->peak_val = bv;
        out->peak_idx = bi;
        out->nx2 = momx[1];
        out->ny2 = momy[1];
    }
}

// ------------------------------------------------------------- launchers --
static inline unsigned ew_blocks(long long n, int num_sms) {
    long long b = (n + 255) / 256;
    const long long cap = (long long)num_sms * 8;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

cudaError_t launch_divide(const float *num, const float *den, long long hw, int C, int gray, float *K, int sms,
                          cudaStream_t st) {
    k_divide<<<ew_blocks(hw, sms), 256, 0, st>>>(num, den, hw, C, gray, K);
    return cudaGetLastError();
}

cudaError_t launch_zero_mean(float *K, int H, int W, double *colmean, double *rowmean, int sms, cudaStream_t st) {
    k_colmean<<<(W + 255) / 256, 256, 0, st>>>(K, H, W, colmean);
    k_rowmean<<<H, RB, 0, st>>>(K, H, W, colmean, rowmean);
    k_sub_means<<<ew_blocks((long long)H * W, sms), 256, 0, st>>>(K, H, W, colmean, rowmean);
    return cudaGetLastError();
}

// out[0] = mean, out[1] = variance (population); two passes about the mean
cudaError_t launch_mean_var(const float *v, long long n, double *part, int nb, double *tmp, double *out,
                            cudaStream_t st) {
    k_moments<<<nb, RB, 0, st>>>(v, n, nullptr, part);
    k_moments_final<<<1, RB, 0, st>>>(part, nb, n, nullptr, tmp);
    k_moments<<<nb, RB, 0, st>>>(v, n, tmp, part);
    k_moments_final<<<1, RB, 0, st>>>(part, nb, n, tmp, out);
    // out[0] = tmp[0] + mean of deviations (a refinement of the mean)
    return cudaGetLastError();
}

cudaError_t launch_to_complex(const float *K, long long n, cufftComplex *F, int sms, cudaStream_t st) {
    k_to_complex<<<ew_blocks(n, sms), 256, 0, st>>>(K, n, F);
    return cudaGetLastError();
}
cudaError_t launch_magnitude(const cufftComplex *F, long long n, float inv_sqrt_n, float *M, int sms,
                             cudaStream_t st) {
    k_magnitude<<<ew_blocks(n, sms), 256, 0, st>>>(F, n, inv_sqrt_n, M);
    return cudaGetLastError();
}
cudaError_t launch_apply_ratio(cufftComplex *F, const float *M, const float *Mn, long long n, int sms,
                               cudaStream_t st) {
    k_apply_ratio<<<ew_blocks(n, sms), 256, 0, st>>>(F, M, Mn, n);
    return cudaGetLastError();
}
cudaError_t launch_real_scaled(const cufftComplex *F, long long n, float scale, float *K, int sms,
                               cudaStream_t st) {
    k_real_scaled<<<ew_blocks(n, sms), 256, 0, st>>>(F, n, scale, K);
    return cudaGetLastError();
}
cudaError_t launch_pce_prep(const float *K, const float *Wq, const float *Iq, long long hw, int C, float *X,
                            float *Y, int sms, cudaStream_t st) {
    k_pce_prep<<<ew_blocks(hw, sms), 256, 0, st>>>(K, Wq, Iq, hw, C, X, Y);
    return cudaGetLastError();
}
cudaError_t launch_sub_center(float *v, long long n, const double *mean, int sms, cudaStream_t st) {
    k_sub_center<<<ew_blocks(n, sms), 256, 0, st>>>(v, n, mean);
    return cudaGetLastError();
}
cudaError_t launch_cross_spectrum(const cufftComplex *FX, const cufftComplex *FY, long long n, cufftComplex *Z,
                                  int sms, cudaStream_t st) {
    k_cross_spectrum<<<ew_blocks(n, sms), 256, 0, st>>>(FX, FY, n, Z);
    return cudaGetLastError();
}
cudaError_t launch_pce_reduce(const float *Cr, int H, int W, int r, int nb, double *part_e, float *part_v,
                              long long *part_i, const double *momx, const double *momy, void *out,
                              cudaStream_t st) {
    k_pce_energy<<<nb, RB, 0, st>>>(Cr, H, W, r, part_e, part_v, part_i);
    k_pce_final<<<1, RB, 0, st>>>(Cr, part_e, part_v, part_i, nb, momx, momy, (PceScalars *)out);
    return cudaGetLastError();
}

size_t pce_scalars_bytes() { return sizeof(PceScalars); }

void pce_unpack(const void *p, double *c0, double *energy, long long *peak_idx, double *nx2, double *ny2) {
    const PceScalars *s = (const PceScalars *)p;
    *c0 = s->c0;
    *energy = s->energy;
    *peak_idx = s->peak_idx;
    *nx2 = s->nx2;
    *ny2 = s->ny2;
}

}  // namespace prnu
