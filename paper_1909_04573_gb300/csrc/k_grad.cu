// k_grad.cu -- adjoint (vector-Jacobian) kernels of the extraction chain with
// free per-frame SDA weights and a differentiable sigma0:
//   S_i = sum_{j in group i} w_j I_j                 (Sec. III-B)
//   W_i = residual(S_i; sigma0)                      (Sec. II-A / III-A)
//   K   = sum_i W_i S_i / sum_i S_i^2                (Sec. III-A)
//   PCE of queries against K                         (Sec. IV)
// The residual's adjoint reuses the forward DWT kernels (the periodised
// orthonormal transform's transpose is its inverse); the shrink's adjoint and
// the other steps are here.
#include <algorithm>

#include "kernels.cuh"

namespace prnu {

// ------------------------------------------------------- weighted SDA -----
// S[g][c][y][x] = sum over the group's frames j of w[j] * I_j[y][x][c], in
// float32 (fma in frame order).  Same blocking as the SDA sum: a block owns a
// row segment of SEGPX pixels of one group, a thread one 16-byte chunk.
template <int C, int SEGPX>
__global__ void __launch_bounds__(SEGPX * C / 16) k_sda_weighted(SdaArgs a, const float *wts) {
    constexpr int NT = SEGPX * C / 16;
    __shared__ float sbuf[SEGPX * C];
    const int rowbytes = a.W * C;
    const int nseg = (a.W + SEGPX - 1) / SEGPX;
    const long long units = (long long)a.G * a.H * nseg;
    const long long plane = (long long)a.H * a.W;
    const int k = threadIdx.x;
    const bool al16 = ((reinterpret_cast<uintptr_t>(a.frames) | (uintptr_t)a.frame_stride | (uintptr_t)a.row_pitch) &
                       15u) == 0;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        const int seg = (int)(u % nseg);
        const long long r = u / nseg;
        const int y = (int)(r % a.H);
        const int gi = (int)(r / a.H);
        const int j0 = (a.g0 + gi) * a.d, j1 = min(a.m, j0 + a.d);
        const int x0 = seg * SEGPX;
        const int npx = min(SEGPX, a.W - x0);
        const int b0 = x0 * C + 16 * k;
        const int nb = min(16, rowbytes - b0);
        float acc[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[i] = 0.f;
        if (nb > 0) {
            const uint8_t *base = a.frames + (long long)y * a.row_pitch + b0;
            if (al16 && nb == 16) {
                for (int j = j0; j < j1; ++j) {
                    const float w = __ldg(wts + j);
                    const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(base + (long long)j * a.frame_stride));
                    const uint32_t wd[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q)
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            acc[4 * q + e] = __fmaf_rn(w, (float)((wd[q] >> (8 * e)) & 0xFFu), acc[4 * q + e]);
                }
            } else {
                for (int j = j0; j < j1; ++j) {
                    const float w = __ldg(wts + j);
                    const uint8_t *p = base + (long long)j * a.frame_stride;
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (i < nb) acc[i] = __fmaf_rn(w, (float)p[i], acc[i]);
                }
            }
        }
        if (u != blockIdx.x) __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) sbuf[16 * k + i] = acc[i];
        __syncthreads();
        float *o = a.out + (long long)gi * C * plane + (long long)y * a.W + x0;
#pragma unroll
        for (int c = 0; c < C; ++c)
            for (int x = k; x < npx; x += NT) o[(long long)c * plane + x] = sbuf[x * C + c];
    }
}

cudaError_t launch_sda_weighted(const SdaArgs &a, const float *wts, int num_sms, cudaStream_t st) {
    if (a.C == 3) {
        constexpr int SEG = 1024, NT = SEG * 3 / 16;
        const long long units = (long long)a.G * a.H * ((a.W + SEG - 1) / SEG);
        const long long blocks = std::max<long long>(1, std::min<long long>(units, (long long)num_sms * (2048 / NT)));
        k_sda_weighted<3, SEG><<<(unsigned)blocks, NT, 0, st>>>(a, wts);
    } else {
        constexpr int SEG = 4096, NT = SEG / 16;
        const long long units = (long long)a.G * a.H * ((a.W + SEG - 1) / SEG);
        const long long blocks = std::max<long long>(1, std::min<long long>(units, (long long)num_sms * (2048 / NT)));
        k_sda_weighted<1, SEG><<<(unsigned)blocks, NT, 0, st>>>(a, wts);
    }
    return cudaGetLastError();
}

// d/dw_j = <gS_{group(j)}, I_j>: block b of frame j sums rows b, b + nb, ...
// into part[j][b] (float64); a second kernel adds the nb parts in order.
constexpr int WG_THREADS = 256;

// Sum over the block (all threads call it); tid is the linear thread index
// and nthreads the block size (a multiple of 32).  Thread 0 gets the total.
__device__ __forceinline__ double block_sum_d(double v, double *sh, int tid, int nthreads) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = tid & 31, wid = tid >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = tid < (nthreads >> 5) ? sh[lane] : 0.0;
    if (wid == 0)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(WG_THREADS) k_sda_wgrad_part(SdaArgs a, const float *gS, double *part) {
    __shared__ double sh[32];
    const int j = blockIdx.y;
    const int gi = j / a.d;
    const long long plane = (long long)a.H * a.W;
    const float *g = gS + (long long)gi * a.C * plane;
    const int rowbytes = a.W * a.C;
    float acc = 0.f;
    for (int y = blockIdx.x; y < a.H; y += gridDim.x) {
        const uint8_t *row = a.frames + (long long)j * a.frame_stride + (long long)y * a.row_pitch;
        const float *grow = g + (long long)y * a.W;
        for (int b = threadIdx.x; b < rowbytes; b += blockDim.x) {
            const int x = b / a.C, c = b - x * a.C;
            acc = __fmaf_rn((float)row[b], __ldg(grow + (long long)c * plane + x), acc);
        }
    }
    const double s = block_sum_d((double)acc, sh, threadIdx.x, blockDim.x);
    if (threadIdx.x == 0) part[(long long)j * gridDim.x + blockIdx.x] = s;
}

__global__ void k_sda_wgrad_final(const double *part, int nb, int m, float *gw) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(long long)j * nb + b];
    gw[j] = (float)s;
}

int sda_wgrad_blocks(int H) { return std::min(H, 64); }

cudaError_t launch_sda_wgrad(const SdaArgs &a, const float *gS, double *part, float *gw, cudaStream_t st) {
    const int nb = sda_wgrad_blocks(a.H);
    k_sda_wgrad_part<<<dim3(nb, a.m), WG_THREADS, 0, st>>>(a, gS, part);
    k_sda_wgrad_final<<<(a.m + 127) / 128, 128, 0, st>>>(part, nb, a.m, gw);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ MLE ----
// num = sum_i W_i S_i, den = sum_i S_i^2 per pixel-channel (fma in image
// order), K = num / den (0 where den == 0), optionally grey (0.299/0.587/0.114).
__global__ void k_mle_images(const float *res, const float *img, int n, int C, long long hw, int gray, float *num,
                             float *den, float *K) {
    const float wg[3] = {0.299f, 0.587f, 0.114f};
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < hw;
         x += (long long)gridDim.x * blockDim.x) {
        float kg = 0.f;
        for (int c = 0; c < C; ++c) {
            float nm = 0.f, dn = 0.f;
            for (int i = 0; i < n; ++i) {
                const long long o = ((long long)i * C + c) * hw + x;
                const float s = __ldg(img + o);
                nm = __fmaf_rn(__ldg(res + o), s, nm);
                dn = __fmaf_rn(s, s, dn);
            }
            num[c * hw + x] = nm;
            den[c * hw + x] = dn;
            const float k = dn != 0.f ? __fdiv_rn(nm, dn) : 0.f;
            if (gray)
                kg = C == 3 ? __fmaf_rn(wg[c], k, kg) : k;
            else
                K[c * hw + x] = k;
        }
        if (gray) K[x] = kg;
    }
}

// g_num = gK / den, g_den = -gK num / den^2; gW_i = g_num S_i,
// gS_i = g_num W_i + 2 g_den S_i (both written).
__global__ void k_mle_images_bwd(const float *res, const float *img, int n, int C, long long hw, int gray,
                                 const float *num, const float *den, const float *gK, float *gres, float *gimg) {
    const float wg[3] = {0.299f, 0.587f, 0.114f};
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < hw;
         x += (long long)gridDim.x * blockDim.x) {
        for (int c = 0; c < C; ++c) {
            const float gk = gray ? (C == 3 ? wg[c] : 1.f) * gK[x] : gK[c * hw + x];
            const float dn = den[c * hw + x];
            float gn = 0.f, gd = 0.f;
            if (dn != 0.f) {
                gn = __fdiv_rn(gk, dn);
                gd = -__fdiv_rn(gn * num[c * hw + x], dn);
            }
            for (int i = 0; i < n; ++i) {
                const long long o = ((long long)i * C + c) * hw + x;
                const float s = __ldg(img + o);
                gres[o] = gn * s;
                gimg[o] = __fmaf_rn(gn, __ldg(res + o), 2.f * gd * s);
            }
        }
    }
}

static inline unsigned ew_grid(long long n, int sms) {
    const long long b = (n + 255) / 256;
    return (unsigned)std::max<long long>(1, std::min<long long>(b, (long long)sms * 8));
}

cudaError_t launch_mle_images(const float *res, const float *img, int n, int C, long long hw, int gray, float *num,
                              float *den, float *K, int sms, cudaStream_t st) {
    k_mle_images<<<ew_grid(hw, sms), 256, 0, st>>>(res, img, n, C, hw, gray, num, den, K);
    return cudaGetLastError();
}

cudaError_t launch_mle_images_bwd(const float *res, const float *img, int n, int C, long long hw, int gray,
                                  const float *num, const float *den, const float *gK, float *gres, float *gimg,
                                  int sms, cudaStream_t st) {
    k_mle_images_bwd<<<ew_grid(hw, sms), 256, 0, st>>>(res, img, n, C, hw, gray, num, den, gK, gres, gimg);
    return cudaGetLastError();
}

// --------------------------------------------------------- shrink adjoint --
// Forward (per subband sample p): m(p) = min_w (1/w^2) sum_{q in w x w(p)}
// c(q)^2 (periodic), den = max(0, m - s2) + s2, n = c s2 / den.  Given gn:
//   active (m > s2):  n = c s2 / m
//     gc(p)  += gn(p) s2 / m(p)                         (direct)
//     gm(p)   = -gn(p) c(p) s2 / m(p)^2
//     gc(q)  += 2 c(q) sum_{p : q in window w*(p) of p} gm(p) / w*(p)^2
//     gs2    += gn(p) c(p) / m(p)     (g_sigma0 += 2 sigma0 gs2)
//   otherwise n = c (s2 > 0): gc(p) += gn(p).
// w*(p) is the first window attaining the minimum (ties: the smaller window).
// A 32 x 32 output tile needs m, w* and gm on a 4-sample halo, and those need
// c on an 8-sample halo.  Shared memory (dynamic):
//   cb[48][49]   c on the 8-halo
//   rs[4][48][40] row sums of c^2 (then re-used for row sums of gm / w^2)
//   am[40][41]  gm / w*^2 on the 4-halo, wk[40][41] the index of w*
//   dir[32][33] the direct term of the tile
constexpr int GT = 32, GH2 = 8, GH1 = 4, GE1 = GT + 2 * GH2, GE2 = GT + 2 * GH1;
constexpr size_t kShrinkBwdSmem = (size_t)GE1 * (GE1 + 1) * 4 + (size_t)4 * GE1 * GE2 * 4 +
                                  (size_t)GE2 * (GE2 + 1) * 4 + (size_t)GT * (GT + 1) * 4 +
                                  (size_t)GE2 * (GE2 + 1);

__global__ void __launch_bounds__(256) k_shrink_bwd(ShrinkBwdArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    float(*cb)[GE1 + 1] = reinterpret_cast<float(*)[GE1 + 1]>(smem);
    float *rsb = reinterpret_cast<float *>(smem + (size_t)GE1 * (GE1 + 1) * 4);
    float(*am)[GE2 + 1] = reinterpret_cast<float(*)[GE2 + 1]>(rsb + 4 * GE1 * GE2);
    float(*dir)[GT + 1] = reinterpret_cast<float(*)[GT + 1]>(&am[GE2][0]);
    signed char(*wk)[GE2 + 1] = reinterpret_cast<signed char(*)[GE2 + 1]>(&dir[GT][0]);
    __shared__ double sh[32];

    const int plane = blockIdx.z;
    const int y0 = blockIdx.y * GT, x0 = blockIdx.x * GT;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const long long poff = (long long)plane * a.R * a.Cc;
    const float *c = a.c + poff;
    const float *gn = a.gn + poff;
    const float s2 = a.s2;

    for (int i = tid; i < GE1 * GE1; i += 256) {
        const int r = i / GE1, q = i - r * GE1;
        const int gy = wrap_near(y0 + r - GH2, a.R), gx = wrap_near(x0 + q - GH2, a.Cc);
        cb[r][q] = __ldg(c + (long long)gy * a.Cc + gx);
    }
    __syncthreads();
    // row sums of c^2 over the 48 rows, for the 40 columns of the 4-halo
    for (int i = tid; i < GE1 * GE2; i += 256) {
        const int r = i / GE2, q = i - r * GE2;
        for (int w = 0; w < a.win.n; ++w) {
            const int rad = a.win.r[w];
            float s = 0.f;
            for (int dx = -rad; dx <= rad; ++dx) {
                const float v = cb[r][q + GH1 + dx];
                s = __fmaf_rn(v, v, s);
            }
            rsb[(w * GE1 + r) * GE2 + q] = s;
        }
    }
    __syncthreads();
    // m, w*, gm on the 4-halo; direct term and the sigma0 sum on the tile
    float gs = 0.f;
    for (int i = tid; i < GE2 * GE2; i += 256) {
        const int r = i / GE2, q = i - r * GE2;
        float m = __int_as_float(0x7f800000);
        int kmin = 0;
        for (int w = 0; w < a.win.n; ++w) {
            const int rad = a.win.r[w];
            float s = 0.f;
            for (int dy = -rad; dy <= rad; ++dy) s += rsb[(w * GE1 + r + GH1 + dy) * GE2 + q];
            const float mw = s * a.win.inv[w];
            if (mw < m) {
                m = mw;
                kmin = w;
            }
        }
        const float cv = cb[r + GH1][q + GH1];
        const int gy = wrap_near(y0 + r - GH1, a.R), gx = wrap_near(x0 + q - GH1, a.Cc);
        const float g = __ldg(gn + (long long)gy * a.Cc + gx);
        const bool active = m > s2;
        am[r][q] = active ? -g * cv * s2 / (m * m) * a.win.inv[kmin] : 0.f;
        wk[r][q] = (signed char)kmin;
        const int ty = r - GH1, tx = q - GH1;
        if (ty >= 0 && ty < GT && tx >= 0 && tx < GT) {
            const float den = fmaxf(0.f, m - s2) + s2;
            dir[ty][tx] = den > 0.f ? g * (s2 / den) : 0.f;
            if (active && y0 + ty < a.R && x0 + tx < a.Cc) gs = __fmaf_rn(g, cv / m, gs);
        }
    }
    __syncthreads();
    // row sums of gm / w*^2 per window class over the 40 rows, tile columns
    for (int i = tid; i < GE2 * GT; i += 256) {
        const int r = i / GT, q = i - r * GT;
        for (int w = 0; w < a.win.n; ++w) {
            const int rad = a.win.r[w];
            float s = 0.f;
            for (int dx = -rad; dx <= rad; ++dx) {
                const int qq = q + GH1 + dx;
                if (wk[r][qq] == w) s += am[r][qq];
            }
            rsb[(w * GE2 + r) * GT + q] = s;
        }
    }
    __syncthreads();
    for (int i = tid; i < GT * GT; i += 256) {
        const int r = i / GT, q = i - r * GT;
        const int gy = y0 + r, gx = x0 + q;
        if (gy >= a.R || gx >= a.Cc) continue;
        float s = 0.f;
        for (int w = 0; w < a.win.n; ++w) {
            const int rad = a.win.r[w];
            for (int dy = -rad; dy <= rad; ++dy) s += rsb[(w * GE2 + r + GH1 + dy) * GT + q];
        }
        const float cv = cb[r + GH2][q + GH2];
        a.gc[poff + (long long)gy * a.Cc + gx] = __fmaf_rn(2.f * cv, s, dir[r][q]);
    }
    const double tot = block_sum_d((double)gs, sh, tid, 256);
    if (tid == 0 && a.g_sigma && tot != 0.0) atomicAdd(a.g_sigma, (double)a.two_sigma0 * tot);
}

cudaError_t launch_shrink_bwd(const ShrinkBwdArgs &a, cudaStream_t st) {
    // above the 48 KB default: opt in (a host-side attribute of the current device)
    cudaError_t e = cudaFuncSetAttribute(k_shrink_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kShrinkBwdSmem);
    if (e != cudaSuccess) return e;
    dim3 block(32, 8);
    dim3 grid((unsigned)((a.Cc + GT - 1) / GT), (unsigned)((a.R + GT - 1) / GT), (unsigned)a.nplanes);
    k_shrink_bwd<<<grid, block, kShrinkBwdSmem, st>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------ PCE adjoint --
// Cr = N C~ (unnormalised inverse FFT), c0 = Cr[0], energy = sum outside the
// neighbourhood of Cr^2 = N^2 E~, PCE = sign(c0) c0^2 O / energy with O the
// number of samples outside.  dPCE/dC~(s) in units where the later inverse
// FFTs are also unnormalised:
//   G(0) = 2 |c0| O N / energy,  G(s) = -2 PCE N Cr(s) / energy outside, 0 inside.
// G overwrites Cr; each query's G is scaled by its upstream gradient g[q].
__global__ void k_pce_gfield(float *Cr, int H, int W, int r, const PceScalars *scal, const double *g) {
    const int q = blockIdx.y;
    const long long n = (long long)H * W;
    const PceScalars s = scal[q];
    const double O = (double)n - (double)(2 * r + 1) * (2 * r + 1);
    double a0 = 0.0, b = 0.0;
    if (s.energy > 0.0) {
        const double pce = (s.c0 >= 0 ? 1.0 : -1.0) * s.c0 * s.c0 * O / s.energy;
        a0 = 2.0 * g[q] * fabs(s.c0) * O * (double)n / s.energy;
        b = -2.0 * g[q] * pce * (double)n / s.energy;
    }
    const float fb = (float)b;
    float *c = Cr + (long long)q * n;
    for (int y = blockIdx.x; y < H; y += gridDim.x) {
        const bool ynear = min(y, H - y) <= r;
        float *row = c + (long long)y * W;
        for (int x = threadIdx.x; x < W; x += blockDim.x) {
            const bool near = ynear && min(x, W - x) <= r;
            row[x] = (y == 0 && x == 0) ? (float)a0 : (near ? 0.f : fb * row[x]);
        }
    }
}

// B = FG * FX (-> FX slot), A = conj(FG) * FY (-> FY slot); DC bins 0 (the
// forward removed the means by zeroing them).
__global__ void k_pce_spectra_bwd(cufftComplex *FX, cufftComplex *FY, const cufftComplex *FG, long long nh, int n) {
    const long long tot = nh * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        if (i % nh == 0) {
            FX[i] = make_cuFloatComplex(0.f, 0.f);
            FY[i] = make_cuFloatComplex(0.f, 0.f);
            continue;
        }
        const cufftComplex x = FX[i], y = FY[i], gq = FG[i];
        FX[i] = make_cuFloatComplex(gq.x * x.x - gq.y * x.y, gq.x * x.y + gq.y * x.x);
        FY[i] = make_cuFloatComplex(gq.x * y.x + gq.y * y.y, gq.x * y.y - gq.y * y.x);
    }
}

// gY_raw = N dPCE/dY, gX_raw = N dPCE/dX (unnormalised inverse transforms):
// g_res[q][c] = w_c gX_raw / N; g_K = sum_q (or per query) gY_raw / N * grey(I_q).
__global__ void k_pce_bwd_out(const float *gYraw, const float *gXraw, const float *Iq, int n, int C, long long hw,
                              float inv_n, int per_query, float *gK, float *gres) {
    const float wg[3] = {0.299f, 0.587f, 0.114f};
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < hw;
         x += (long long)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int q = 0; q < n; ++q) {
            const float gx = gXraw[(long long)q * hw + x] * inv_n;
            const float gy = gYraw[(long long)q * hw + x] * inv_n;
            const float *im = Iq + (long long)q * C * hw;
            float ig;
            if (C == 3) {
                ig = __fmaf_rn(0.114f, im[2 * hw + x], __fmaf_rn(0.587f, im[hw + x], 0.299f * im[x]));
                for (int c = 0; c < 3; ++c) gres[((long long)q * 3 + c) * hw + x] = wg[c] * gx;
            } else {
                ig = im[x];
                gres[(long long)q * hw + x] = gx;
            }
            if (per_query)
                gK[(long long)q * hw + x] = gy * ig;
            else
                acc = __fmaf_rn(gy, ig, acc);
        }
        if (!per_query) gK[x] = acc;
    }
}

cudaError_t launch_pce_gfield(float *Cr, int H, int W, int r, int n, const void *scal, const double *g,
                              cudaStream_t st) {
    k_pce_gfield<<<dim3(std::min(H, 256), n), 256, 0, st>>>(Cr, H, W, r, static_cast<const PceScalars *>(scal), g);
    return cudaGetLastError();
}

cudaError_t launch_pce_spectra_bwd(cufftComplex *FX, cufftComplex *FY, const cufftComplex *FG, long long nh, int n,
                                   int sms, cudaStream_t st) {
    k_pce_spectra_bwd<<<ew_grid(nh * n, sms), 256, 0, st>>>(FX, FY, FG, nh, n);
    return cudaGetLastError();
}

cudaError_t launch_pce_bwd_out(const float *gYraw, const float *gXraw, const float *Iq, int n, int C, long long hw,
                               float inv_n, int per_query, float *gK, float *gres, int sms, cudaStream_t st) {
    k_pce_bwd_out<<<ew_grid(hw, sms), 256, 0, st>>>(gYraw, gXraw, Iq, n, C, hw, inv_n, per_query, gK, gres);
    return cudaGetLastError();
}

}  // namespace prnu
