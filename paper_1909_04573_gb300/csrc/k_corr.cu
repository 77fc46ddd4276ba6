// Circular cross-correlation of the PCE test (Sec. IV) by our own mixed-radix
// FFTs, fused so that the spectra pass through HBM as few times as possible:
//
//   1. k_rfft_rows     one real FFT per row of X_i and Y_i (length W, as a
//                      complex FFT of length W/2 plus the split step), half
//                      spectra to a padded complex workspace;
//   2. k_corr_columns  per query and tile of spectrum columns: the column FFTs
//                      of X^ and Y^, the cross spectrum conj(X^) Y^ with its
//                      DC bin zeroed (the means removed), and the inverse
//                      column FFT, all in shared memory; the result replaces X^;
//   3. k_corr_rows     per row: the inverse real FFT (the split step, then a
//                      complex FFT of length W/2) and, on the correlation row
//                      it leaves in shared memory, the PCE reductions: energy
//                      outside the (2r+1)^2 neighbourhood of zero shift, the
//                      argmax (first index on ties) and C(0, 0).
//
// The correlation plane itself is never written.  All transforms are
// unnormalised (the result is H*W times the correlation), like cuFFT's.
//
// Each 1-D transform is a Stockham autosort FFT over the factors 8, 4, 2, 9,
// 15, 3, 5, 7 of its length (9 and 15 as register-resident composite
// butterflies); one pass per factor, ping-ponging between two shared
// buffers.  Several sequences are interleaved element by element and
// consecutive threads take consecutive sequences; rows of the interleaved
// layout are padded (at<G>) so that the strided writes of the early passes
// spread over the banks too.  Twiddles are computed once per call in float64
// (k_twiddles) and rounded to float.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "kernels.cuh"

namespace prnu {
namespace {

constexpr int CT = 256;    // threads per block of the inverse row pass (its registers allow no more)
constexpr int CTH = 544;   // threads of the column pass of 1080-point columns: its first (radix-8)
                           // pass over two columns of X^ and Y^ has 540 butterflies, one per thread
constexpr int CTW = 512;   // threads per block of the forward row and the column passes: their shared
                           // memory allows two blocks per SM, so twice the threads double the warps

// complex arithmetic on {re, im} as packed float32x2 (each lane round-to-nearest)
__device__ __forceinline__ pf2 pk(float2 a) { return pf2_of(a.x, a.y); }
__device__ __forceinline__ float2 upk(pf2 v) {
    float2 r;
    pf2_split(v, r.x, r.y);
    return r;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
    pf2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
    return upk(r);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
    pf2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
    return upk(r);
}
// a b = {a.x b.x - a.y b.y, a.x b.y + a.y b.x}: {-a.y b.y, a.y b.x}, then one packed FMA
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    pf2 p;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(p) : "l"(pf2_of(-a.y, a.y)), "l"(pf2_of(b.y, b.x)));
    return upk(pf2_fma(pf2_of(a.x, a.x), pk(b), p));
}
__device__ __forceinline__ float2 cmi(float2 a) { return make_float2(a.y, -a.x); }  // -i a
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// ---------------------------------------------------------- small DFTs ---
// Forward (exponent sign -1), in registers.
template <int R>
struct Dft;

template <>
struct Dft<2> {
    static __device__ __forceinline__ void run(float2 *v) {
        const float2 t = v[0];
        v[0] = cadd(t, v[1]);
        v[1] = csub(t, v[1]);
    }
};

template <>
struct Dft<4> {
    static __device__ __forceinline__ void run(float2 *v) {
        const float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        const float2 s13 = cadd(v[1], v[3]), d13 = cmi(csub(v[1], v[3]));
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, d13);
        v[3] = csub(d02, d13);
    }
};

template <>
struct Dft<8> {
    static __device__ __forceinline__ void run(float2 *v) {
        constexpr float h = 0.70710678118654752f;  // sqrt(1/2)
        float2 e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4>::run(e);
        Dft<4>::run(o);
        o[1] = make_float2((o[1].x + o[1].y) * h, (o[1].y - o[1].x) * h);   // * e^{-i pi/4}
        o[2] = cmi(o[2]);                                                   // * e^{-i pi/2}
        o[3] = make_float2((o[3].y - o[3].x) * h, -(o[3].x + o[3].y) * h);  // * e^{-3i pi/4}
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = cadd(e[k], o[k]);
            v[k + 4] = csub(e[k], o[k]);
        }
    }
};

template <>
struct Dft<3> {
    static __device__ __forceinline__ void run(float2 *v) {
        constexpr float c = 0.86602540378443865f;  // sin(2 pi / 3)
        const float2 s = cadd(v[1], v[2]), d = cmi(csub(v[1], v[2]));
        const float2 t = make_float2(__fmaf_rn(-0.5f, s.x, v[0].x), __fmaf_rn(-0.5f, s.y, v[0].y));
        v[0] = cadd(v[0], s);
        v[1] = make_float2(__fmaf_rn(c, d.x, t.x), __fmaf_rn(c, d.y, t.y));
        v[2] = make_float2(__fmaf_rn(-c, d.x, t.x), __fmaf_rn(-c, d.y, t.y));
    }
};

// odd prime R: y_k = v_0 + sum_{m=1}^{(R-1)/2} [(v_m + v_{R-m}) cos(2 pi m k / R)
//                                             - i (v_m - v_{R-m}) sin(2 pi m k / R)]
// and y_{R-k} the same with +i; cos/sin of 2 pi q / R for q = 0..(R-1)/2.
template <int R>
struct OddConst;
template <>
struct OddConst<5> {
    static __device__ __forceinline__ float c(int q) {
        return q == 0 ? 1.f : (q == 1 ? 0.30901699437494742f : -0.80901699437494742f);
    }
    static __device__ __forceinline__ float s(int q) {
        return q == 0 ? 0.f : (q == 1 ? 0.95105651629515357f : 0.58778525229247313f);
    }
};
template <>
struct OddConst<7> {
    static __device__ __forceinline__ float c(int q) {
        return q == 0 ? 1.f
                      : (q == 1 ? 0.62348980185873353f : (q == 2 ? -0.22252093395631440f : -0.90096886790241913f));
    }
    static __device__ __forceinline__ float s(int q) {
        return q == 0 ? 0.f : (q == 1 ? 0.78183148246802981f : (q == 2 ? 0.97492791218182361f : 0.43388373911755812f));
    }
};

template <int R>
struct DftOdd {
    static __device__ __forceinline__ void run(float2 *v) {
        constexpr int H = (R - 1) / 2;
        float2 A[H + 1], B[H + 1];
#pragma unroll
        for (int m = 1; m <= H; ++m) {
            A[m] = cadd(v[m], v[R - m]);
            B[m] = cmi(csub(v[m], v[R - m]));  // -i (v_m - v_{R-m})
        }
        float2 y0 = v[0];
#pragma unroll
        for (int m = 1; m <= H; ++m) y0 = cadd(y0, A[m]);
        float2 out[R];
        out[0] = y0;
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            float2 re = v[0], im = make_float2(0.f, 0.f);
#pragma unroll
            for (int m = 1; m <= H; ++m) {
                const int idx = (m * k) % R;
                const int q = idx <= H ? idx : R - idx;
                const float cs = OddConst<R>::c(q);
                const float sn = idx <= H ? OddConst<R>::s(q) : -OddConst<R>::s(q);
                re = make_float2(__fmaf_rn(cs, A[m].x, re.x), __fmaf_rn(cs, A[m].y, re.y));
                im = make_float2(__fmaf_rn(sn, B[m].x, im.x), __fmaf_rn(sn, B[m].y, im.y));
            }
            out[k] = cadd(re, im);
            out[R - k] = csub(re, im);
        }
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = out[k];
    }
};
template <>
struct Dft<5> : DftOdd<5> {};
template <>
struct Dft<7> : DftOdd<7> {};

// 9 = 3 x 3 (Cooley-Tukey, twiddles w_9^{n2 k1} as constants):
// X[k1 + 3 k2] = sum_n2 w_3^{n2 k2} w_9^{n2 k1} sum_n1 x[3 n1 + n2] w_3^{n1 k1}
template <>
struct Dft<9> {
    static __device__ __forceinline__ void run(float2 *v) {
        // w_9^j = (cos 2 pi j / 9, -sin 2 pi j / 9), j = 1, 2, 4
        const float2 w1 = make_float2(0.76604444311897804f, -0.64278760968653933f);
        const float2 w2 = make_float2(0.17364817766693035f, -0.98480775301220806f);
        const float2 w4 = make_float2(-0.93969262078590838f, -0.34202014332566873f);
        float2 y[3][3];
#pragma unroll
        for (int n2 = 0; n2 < 3; ++n2) {
            float2 a[3] = {v[n2], v[3 + n2], v[6 + n2]};
            Dft<3>::run(a);
            y[n2][0] = a[0];
            y[n2][1] = n2 == 0 ? a[1] : cmul(a[1], n2 == 1 ? w1 : w2);
            y[n2][2] = n2 == 0 ? a[2] : cmul(a[2], n2 == 1 ? w2 : w4);
        }
#pragma unroll
        for (int k1 = 0; k1 < 3; ++k1) {
            float2 b[3] = {y[0][k1], y[1][k1], y[2][k1]};
            Dft<3>::run(b);
#pragma unroll
            for (int k2 = 0; k2 < 3; ++k2) v[k1 + 3 * k2] = b[k2];
        }
    }
};

// 15 = 3 x 5 by the prime-factor (Good-Thomas) map, no twiddles:
// input n = (5 n1 + 3 n2) mod 15, output k = (10 k1 + 6 k2) mod 15
template <>
struct Dft<15> {
    static __device__ __forceinline__ void run(float2 *v) {
        float2 b[3][5];
#pragma unroll
        for (int n2 = 0; n2 < 5; ++n2) {
            float2 c[3] = {v[(3 * n2) % 15], v[(5 + 3 * n2) % 15], v[(10 + 3 * n2) % 15]};
            Dft<3>::run(c);
#pragma unroll
            for (int k1 = 0; k1 < 3; ++k1) b[k1][n2] = c[k1];
        }
#pragma unroll
        for (int k1 = 0; k1 < 3; ++k1) {
            Dft<5>::run(b[k1]);
#pragma unroll
            for (int k2 = 0; k2 < 5; ++k2) v[(10 * k1 + 6 * k2) % 15] = b[k1][k2];
        }
    }
};

// ------------------------------------------------------ Stockham passes ---
// Element j of interleaved sequence g sits at at<G>(j, g): rows of G
// elements with one row of padding after every 8, so that the strided
// writes of the early passes (stride R rows) spread over the banks as the
// contiguous reads do; padded row prow(j + 8c) = prow(j) + 9c, so offsets
// stay linear in the butterfly's element index wherever the stride is a
// multiple of 8.
__host__ __device__ constexpr int prow(int j) { return j + (j >> 3); }
template <int G>
__device__ __forceinline__ int at(int j, int g) {
    return prow(j) * G + g;
}
__host__ __device__ constexpr int padded_len(int n) { return n + (n >> 3) + 1; }

// twiddles w_L^{m ts} (exponent sign -1, or +1 with INV), then the radix-R DFT
template <int R, bool INV>
__device__ __forceinline__ void butterfly(float2 *v, const float2 *__restrict__ tw, int ts) {
    if (ts) {
#pragma unroll
        for (int m = 1; m < R; ++m) {
            float2 t = tw[m * ts];
            if (INV) t.y = -t.y;
            v[m] = cmul(v[m], t);
        }
    }
    if (INV) {
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = cconj(v[m]);
    }
    Dft<R>::run(v);
    if (INV) {
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = cconj(v[m]);
    }
}

// One radix-R pass over NA sequences of length L in a layout of G
// interleaved sequences, from a to b; Ns = product of the radices already
// applied.  Butterfly j reads elements j + m L/R and writes
// (j - j%Ns) R + j%Ns + m Ns (Stockham autosort).
template <int R, int G, int NA, bool INV>
__device__ __forceinline__ void fft_pass(const float2 *__restrict__ a, float2 *__restrict__ b, int L, int Ns,
                                         const float2 *__restrict__ tw) {
    const int nb = L / R;
    const int step = L / (Ns * R);
    for (int u = threadIdx.x; u < nb * NA; u += blockDim.x) {
        const int g = u % NA, j = u / NA;
        const int k = j % Ns;
        float2 v[R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = a[at<G>(j + m * nb, g)];
        butterfly<R, INV>(v, tw, k * step);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int m = 0; m < R; ++m) b[at<G>(base + m * Ns, g)] = v[m];
    }
}

// All passes for a length known at run time; the input is in a (visible to
// the block), the result in the returned buffer, visible to the block.
template <int G, int NA, bool INV>
__device__ float2 *fft_run(float2 *a, float2 *b, const FftSteps &p, const float2 *tw) {
    int Ns = 1;
    for (int i = 0; i < p.np; ++i) {
        const int R = p.r(i);
        switch (R) {
            case 8: fft_pass<8, G, NA, INV>(a, b, p.L, Ns, tw); break;
            case 4: fft_pass<4, G, NA, INV>(a, b, p.L, Ns, tw); break;
            case 2: fft_pass<2, G, NA, INV>(a, b, p.L, Ns, tw); break;
            case 3: fft_pass<3, G, NA, INV>(a, b, p.L, Ns, tw); break;
            case 5: fft_pass<5, G, NA, INV>(a, b, p.L, Ns, tw); break;
            case 9: fft_pass<9, G, NA, INV>(a, b, p.L, Ns, tw); break;
            case 15: fft_pass<15, G, NA, INV>(a, b, p.L, Ns, tw); break;
            default: fft_pass<7, G, NA, INV>(a, b, p.L, Ns, tw); break;
        }
        __syncthreads();
        float2 *t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

// The same with the length fixed at compile time: the pass sequence, strides
// and loop trip counts are constants (the block has NT threads).
struct StaticPlan {
    int np = 0;
    int r[kMaxFftPasses] = {}, ns[kMaxFftPasses] = {};
};
// Powers of two first (8, 4, 2), then the odd part in register radices 9
// and 15 where they divide it, then 3, 5, 7: 960 = 8.8.15, 1080 = 8.9.15.
__host__ __device__ constexpr StaticPlan static_plan(int L) {
    StaticPlan p{};
    const int rs[8] = {8, 4, 2, 9, 15, 3, 5, 7};
    int x = L, ns = 1;
    for (int i = 0; i < 8; ++i)
        while (x % rs[i] == 0 && p.np < kMaxFftPasses) {
            p.r[p.np] = rs[i];
            p.ns[p.np] = ns;
            ns *= rs[i];
            x /= rs[i];
            ++p.np;
        }
    if (x != 1) p.np = -1;
    return p;
}

template <int R, int L, int Ns, int G, int NA, bool INV, int NT>
__device__ __forceinline__ void fft_pass_s(const float2 *__restrict__ a, float2 *__restrict__ b,
                                           const float2 *__restrict__ tw) {
    constexpr int nb = L / R, step = L / (Ns * R), total = nb * NA;
    // element offsets linear in m: loads when nb is a multiple of 8; stores
    // when Ns is, or when Ns = 1 and R divides 8 (base = j R, m < R)
    constexpr bool ld_lin = nb % 8 == 0;
    constexpr bool st_lin = Ns % 8 == 0 || (Ns == 1 && 8 % R == 0);
    constexpr int ld_step = prow(nb), st_step = Ns == 1 ? 1 : prow(Ns);
#pragma unroll
    for (int it = 0; it < (total + NT - 1) / NT; ++it) {
        const int u = (int)threadIdx.x + it * NT;
        if (total % NT == 0 || u < total) {
            const int g = u % NA, j = u / NA;
            const int k = Ns == 1 ? 0 : j % Ns;
            float2 v[R];
            if constexpr (ld_lin) {
                const float2 *src = a + at<G>(j, g);
#pragma unroll
                for (int m = 0; m < R; ++m) v[m] = src[m * ld_step * G];
            } else {
#pragma unroll
                for (int m = 0; m < R; ++m) v[m] = a[at<G>(j + m * nb, g)];
            }
            butterfly<R, INV>(v, tw, k * step);
            const int base = (j - k) * R + k;
            if constexpr (st_lin) {
                float2 *dst = b + at<G>(base, g);
#pragma unroll
                for (int m = 0; m < R; ++m) dst[m * st_step * G] = v[m];
            } else {
#pragma unroll
                for (int m = 0; m < R; ++m) b[at<G>(base + m * Ns, g)] = v[m];
            }
        }
    }
}

template <int L, int G, int NA, bool INV, int NT, int P = 0>
__device__ __forceinline__ float2 *fft_run_s(float2 *a, float2 *b, const float2 *tw) {
    constexpr StaticPlan pl = static_plan(L);
    static_assert(pl.np > 0, "length must factor into 2, 3, 5, 7");
    if constexpr (P == pl.np) {
        return a;
    } else {
        fft_pass_s<pl.r[P], L, pl.ns[P], G, NA, INV, NT>(a, b, tw);
        __syncthreads();
        return fft_run_s<L, G, NA, INV, NT, P + 1>(b, a, tw);
    }
}

// LS > 0: the length is LS (compile time); else p.L.  NT: threads per block.
template <int LS, int G, int NA, bool INV, int NT>
__device__ __forceinline__ float2 *fft_any(float2 *a, float2 *b, const FftSteps &p, const float2 *tw) {
    if constexpr (LS > 0)
        return fft_run_s<LS, G, NA, INV, NT>(a, b, tw);
    else
        return fft_run<G, NA, INV>(a, b, p, tw);
}

// 8-byte global -> shared copies in flight together (cp.async groups)
__device__ __forceinline__ void cp_async8(float2 *dst, const float2 *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void load_table(float2 *dst, const float2 *__restrict__ src, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// ------------------------------------------------------------- kernels ---
// tw_m[i] = e^{-2 pi i i / M} (i < M), tw_h[k] = e^{-2 pi i k / W} (k <= M),
// tw_c[i] = e^{-2 pi i i / H} (i < H), M = W / 2; float64 then rounded.
__global__ void k_twiddles(float2 *tw, int M, int H) {
    const int n = M + (M + 1) + H;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double a;  // angle / (-pi)
        if (i < M)
            a = 2.0 * i / M;
        else if (i < 2 * M + 1)
            a = (double)(i - M) / M;
        else
            a = 2.0 * (i - 2 * M - 1) / H;
        double s, c;
        sincospi(-a, &s, &c);
        tw[i] = make_float2((float)c, (float)s);
    }
}

// Real FFT of nrows rows of length W (pitch W floats) to half spectra of
// M + 1 bins (pitch ldo complex); G rows per block iteration.  Three buffers
// rotate: the next rows are staged (cp.async) while the current ones are
// transformed in the other two.
template <int G, int MS, int NT>
__global__ void __launch_bounds__(NT) k_rfft_rows(const float *__restrict__ x, float2 *__restrict__ out,
                                                  long long nrows, int W, int ldo, FftSteps p,
                                                  const float2 *__restrict__ twg) {
    extern __shared__ float2 sm[];
    const int M = MS > 0 ? MS : W >> 1;
    float2 *tw = sm;  // w_M^i; the split step's w_W^k are read through L1 (once per element)
    const float2 *__restrict__ twh = twg + M;
    const int BS = G * padded_len(M + 1);
    float2 *const buf0 = sm + M;  // three buffers of BS
    load_table(tw, twg, M);
    auto stage = [&](long long r0, float2 *dst) {
        for (int u = threadIdx.x; u < G * M; u += blockDim.x) {
            const int g = u % G, m = u / G;
            const long long r = r0 + g;
            if (r < nrows)
                cp_async8(dst + at<G>(m, g), reinterpret_cast<const float2 *>(x + r * W) + m);
            else
                dst[at<G>(m, g)] = make_float2(0.f, 0.f);
        }
    };
    const long long stride = (long long)gridDim.x * G;
    long long r0 = (long long)blockIdx.x * G;
    if (r0 < nrows) stage(r0, buf0);
    cp_async_commit();
    for (int i = 0; r0 < nrows; r0 += stride, ++i) {
        float2 *cur = buf0 + (i % 3) * BS, *nxt = buf0 + ((i + 1) % 3) * BS, *scr = buf0 + ((i + 2) % 3) * BS;
        if (r0 + stride < nrows) stage(r0 + stride, nxt);
        cp_async_commit();
        cp_async_wait<1>();  // this iteration's rows have landed
        __syncthreads();
        const float2 *Z = fft_any<MS, G, G, false, NT>(cur, scr, p, tw);
        // split step: X_k = (Z_k + conj Z_{M-k}) / 2 - i w_W^k (Z_k - conj Z_{M-k}) / 2
        for (int u = threadIdx.x; u < G * (M + 1); u += blockDim.x) {
            const int g = u % G, k = u / G;
            const long long r = r0 + g;
            if (r >= nrows) continue;
            const float2 zk = Z[at<G>(k == M ? 0 : k, g)];
            const float2 zc = cconj(Z[at<G>(k == 0 ? 0 : M - k, g)]);
            const float2 s = cadd(zk, zc), wd = cmul(__ldg(twh + k), csub(zk, zc));
            if (PRNU_DCHECK(k < ldo, k)) out[r * ldo + k] = make_float2(0.5f * (s.x + wd.y), 0.5f * (s.y - wd.x));
        }
        __syncthreads();  // cur / scr are restaged from the next iteration on
    }
    cp_async_wait<0>();
}

// Per query q (grid y) and tile of TC spectrum columns (grid x): column FFTs
// of X^_q and Y^_q (F + q*H*ld and F + (n+q)*H*ld, pitch ld), Z = conj(X^) Y^
// with Z(0, 0) = 0, inverse column FFT of Z, written over X^_q.
template <int TC, int HS, int NT>
__global__ void __launch_bounds__(NT) k_corr_columns(float2 *F, int n, int H, int Wh, int ld, FftSteps p,
                                                     const float2 *__restrict__ twg) {
    extern __shared__ float2 sm[];
    constexpr int G = 2 * TC;
    float2 *tw = sm, *A = sm + H, *B = A + G * padded_len(H);
    const int q = blockIdx.y, c0 = blockIdx.x * TC;
    float2 *FX = F + (long long)q * H * ld;
    const float2 *FY = F + (long long)(n + q) * H * ld;
    load_table(tw, twg, H);
    for (int u = threadIdx.x; u < G * H; u += blockDim.x) {
        const int s = u % G, y = u / G, c = c0 + (s < TC ? s : s - TC);
        const float2 *src = s < TC ? FX : FY;
        if (c < Wh && PRNU_DCHECK(c < ld && q < n, c))
            cp_async8(A + at<G>(y, s), src + (long long)y * ld + c);
        else
            A[at<G>(y, s)] = make_float2(0.f, 0.f);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    float2 *S = fft_any<HS, G, G, false, NT>(A, B, p, tw);
    float2 *T = S == A ? B : A;
    // Z into T in its own layout of TC sequences (the inverse then touches
    // whole rows of that layout)
    for (int u = threadIdx.x; u < TC * H; u += blockDim.x) {
        const int s = u % TC, y = u / TC;
        const float2 a = S[at<G>(y, s)], b = S[at<G>(y, TC + s)];
        float2 z = make_float2(__fmaf_rn(a.x, b.x, a.y * b.y), __fmaf_rn(a.x, b.y, -a.y * b.x));
        if (y == 0 && c0 + s == 0) z = make_float2(0.f, 0.f);
        T[at<TC>(y, s)] = z;
    }
    __syncthreads();
    const float2 *Z = fft_any<HS, TC, TC, true, NT>(T, S, p, tw);
    for (int u = threadIdx.x; u < TC * H; u += blockDim.x) {
        const int s = u % TC, y = u / TC, c = c0 + s;
        if (c < Wh && PRNU_DCHECK(c < ld, c)) FX[(long long)y * ld + c] = Z[at<TC>(y, s)];
    }
}

// ------------------------------------------ 1080-point columns, four-step ---
// The column pass of 1080-row planes as a four-step transform held in
// registers, 1080 = 40 x 27 (n = 27 n1 + n2, k = k1 + 40 k2):
//   A[n2][k1] = sum_{n1} x[27 n1 + n2] w_40^{n1 k1}    one thread per n2: a 40-point DFT
//   X[k1 + 40 k2] = sum_{n2} A[n2][k1] w_1080^{n2 k1} w_27^{n2 k2}   one thread per k1: a 27-point DFT
// with one shared-memory transpose between them (the Stockham form moves
// every sample through shared memory once per radix pass, three times).
// The thread of k1 forms both X^ and Y^ there, so the cross spectrum
// Z = conj(X^) Y^ (DC bin zeroed) is made in registers, and it starts the
// inverse right away: with m = k1 + 40 m1, j = j1 + 27 j2,
//   C[k1][j1] = sum_{m1} Z[k1 + 40 m1] w_27^{-m1 j1} w_1080^{-k1 j1}   (27-point, same thread)
//   y[j1 + 27 j2] = sum_{k1} C[k1][j1] w_40^{-k1 j2}                  one thread per j1: 40-point
// The result (unnormalised, as every transform here) replaces X^.
constexpr int K4_N1 = 40, K4_N2 = 27, K4_L = 1080;
constexpr int K4_COLS = 2;                     // spectrum columns per block (4: 0.264 ms, 8: 0.290 ms per
                                               // video step against 0.256 ms; three blocks per SM here)
constexpr int K4_NT = 128;                     // threads: the first step has 2 x 27 x 2 = 108 items
constexpr int K4_SS = K4_N1 * K4_COLS + 4;     // float2 stride of an n2 (or j1) row of the buffers

// 40-point DFT in place, 8 x 5 prime-factor (no twiddles): input index
// (5 a + 8 b) mod 40 -> output index (25 k1 + 16 k2) mod 40
__device__ __forceinline__ void dft40(float2 *v) {
    float2 u[5][8];
#pragma unroll
    for (int b = 0; b < 5; ++b)
#pragma unroll
        for (int a = 0; a < 8; ++a) u[b][a] = v[(5 * a + 8 * b) % 40];
#pragma unroll
    for (int b = 0; b < 5; ++b) Dft<8>::run(u[b]);
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) {
        float2 t[5];
#pragma unroll
        for (int b = 0; b < 5; ++b) t[b] = u[b][k1];
        Dft<5>::run(t);
#pragma unroll
        for (int k2 = 0; k2 < 5; ++k2) v[(25 * k1 + 16 * k2) % 40] = t[k2];
    }
}

// 27-point DFT in place, 3 x 9 with twiddles w_27^m = w_1080^{40 m}
__device__ __forceinline__ void dft27(float2 *v, const float2 *__restrict__ tw) {
    float2 y[3][9];
#pragma unroll
    for (int b = 0; b < 9; ++b) {
        float2 t[3] = {v[b], v[9 + b], v[18 + b]};
        Dft<3>::run(t);
#pragma unroll
        for (int k1 = 0; k1 < 3; ++k1) y[k1][b] = (k1 * b == 0) ? t[k1] : cmul(t[k1], __ldg(tw + 40 * k1 * b));
    }
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) {
        Dft<9>::run(y[k1]);
#pragma unroll
        for (int k2 = 0; k2 < 9; ++k2) v[k1 + 3 * k2] = y[k1][k2];
    }
}

template <int N>
__device__ __forceinline__ void conj_all(float2 *v) {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i].y = -v[i].y;
}

__global__ void __launch_bounds__(K4_NT) k_corr_columns_4s(float2 *F, int n, int Wh, int ld,
                                                           const float2 *__restrict__ tw) {
    extern __shared__ __align__(16) float2 sm4[];
    float2 *S = sm4;                                 // [2][27][K4_SS]: A of X^ and Y^ after the first step
    float2 *T = sm4 + 2 * K4_N2 * K4_SS;             // [27][K4_SS]: C after the first inverse step
    const int q = blockIdx.y, c0 = blockIdx.x * K4_COLS, tid = threadIdx.x;
    float2 *FX = F + (long long)q * K4_L * ld;
    const float2 *FY = F + (long long)(n + q) * K4_L * ld;

    // forward step 1: item (sequence, n2, column)
    if (tid < 2 * K4_N2 * K4_COLS) {
        const int col = tid % K4_COLS, r = tid / K4_COLS, n2 = r % K4_N2, sq = r / K4_N2;
        const int c = c0 + col;
        const float2 *src = (sq ? FY : FX) + c;
        float2 v[K4_N1];
#pragma unroll
        for (int n1 = 0; n1 < K4_N1; ++n1)
            v[n1] = (c < Wh && PRNU_DCHECK(c < ld && q < n, c)) ? src[(long long)(27 * n1 + n2) * ld]
                                                                : make_float2(0.f, 0.f);
        dft40(v);
        float2 *dst = S + (sq * K4_N2 + n2) * K4_SS + col;
#pragma unroll
        for (int k1 = 0; k1 < K4_N1; ++k1)
            dst[k1 * K4_COLS] = (k1 == 0 || n2 == 0) ? v[k1] : cmul(v[k1], __ldg(tw + n2 * k1));
    }
    __syncthreads();
    // forward step 2 and the first inverse step: item (k1, column)
    if (tid < K4_N1 * K4_COLS) {
        const int col = tid % K4_COLS, k1 = tid / K4_COLS;
        float2 a[K4_N2], b[K4_N2];
#pragma unroll
        for (int n2 = 0; n2 < K4_N2; ++n2) {
            a[n2] = S[n2 * K4_SS + k1 * K4_COLS + col];
            b[n2] = S[(K4_N2 + n2) * K4_SS + k1 * K4_COLS + col];
        }
        dft27(a, tw);  // X^[k1 + 40 k2] = a[k2]
        dft27(b, tw);
#pragma unroll
        for (int k2 = 0; k2 < K4_N2; ++k2) {  // Z = conj(X^) Y^, conjugated for the inverse by conjugation
            const float2 x = a[k2], y = b[k2];
            a[k2] = make_float2(__fmaf_rn(x.x, y.x, x.y * y.y), -__fmaf_rn(x.x, y.y, -x.y * y.x));
        }
        if (c0 + col == 0 && k1 == 0) a[0] = make_float2(0.f, 0.f);
        dft27(a, tw);  // conj C (before the inverse twiddle)
        float2 *dst = T + k1 * K4_COLS + col;
#pragma unroll
        for (int j1 = 0; j1 < K4_N2; ++j1) {
            const float2 cj = cconj(a[j1]);
            dst[j1 * K4_SS] = (k1 == 0 || j1 == 0) ? cj : cmul(cj, cconj(__ldg(tw + k1 * j1)));
        }
    }
    __syncthreads();
    // inverse step 2: item (j1, column)
    if (tid < K4_N2 * K4_COLS) {
        const int col = tid % K4_COLS, j1 = tid / K4_COLS;
        const int c = c0 + col;
        float2 v[K4_N1];
#pragma unroll
        for (int k1 = 0; k1 < K4_N1; ++k1) v[k1] = cconj(T[j1 * K4_SS + k1 * K4_COLS + col]);
        dft40(v);
        if (c < Wh && PRNU_DCHECK(c < ld, c)) {
#pragma unroll
            for (int j2 = 0; j2 < K4_N1; ++j2) FX[(long long)(j1 + 27 * j2) * ld + c] = cconj(v[j2]);
        }
    }
}

__device__ __forceinline__ double block_sum_d(double v, double *sh) {
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

// Per query q (grid y): inverse real FFT of rows y = blockIdx.x*G + ... of
// Z_q (pitch ld, M + 1 bins) and the PCE partials of this block: energy
// outside the neighbourhood |dy|, |dx| <= r of zero shift (circular), the
// maximum and its first flat index, and C(0, 0) to c0[q].  The rows are
// staged (cp.async) into one of two buffers while the previous ones are
// transformed in the work buffer and the other.
template <int G, int MS>
__global__ void __launch_bounds__(CT, 3) k_corr_rows(const float2 *__restrict__ Zall, int H, int W, int ld, int r,
                                                  FftSteps p, const float2 *__restrict__ twg, double *part_e,
                                                  float *part_v, long long *part_i, float *c0) {
    extern __shared__ float2 sm[];
    const int M = MS > 0 ? MS : W >> 1, Wh = M + 1;
    float2 *tw = sm, *Wk = sm + M;  // w_M^i; the split step's w_W^k are read through L1
    const float2 *__restrict__ twh = twg + M;
    const int BS = G * padded_len(Wh);
    float2 *const S0 = Wk + BS;  // two staging buffers of BS (G raw rows of Wh bins)
    const int q = blockIdx.y;
    const float2 *Z = Zall + (long long)q * H * ld;
    load_table(tw, twg, M);
    auto stage = [&](int y0, float2 *dst) {
        for (int g = 0; g < G; ++g) {
            const int y = y0 + g;
            for (int k = threadIdx.x; k < Wh; k += blockDim.x) {
                if (y < H && PRNU_DCHECK(k < ld, k))
                    cp_async8(dst + g * Wh + k, Z + (long long)y * ld + k);
                else
                    dst[g * Wh + k] = make_float2(0.f, 0.f);
            }
        }
    };
    double acc = 0.0;
    float bv = -__int_as_float(0x7f800000);
    long long bi = LLONG_MAX;
    const int stride = gridDim.x * G;
    int y0 = blockIdx.x * G;
    if (y0 < H) stage(y0, S0);
    cp_async_commit();
    for (int i = 0; y0 < H; y0 += stride, ++i) {
        float2 *cur = S0 + (i & 1) * BS, *nxt = S0 + ((i + 1) & 1) * BS;
        if (y0 + stride < H) stage(y0 + stride, nxt);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        // split step: Z'_k = E_k + i O_k, E_k = X_k + conj X_{M-k},
        // O_k = (X_k - conj X_{M-k}) e^{+2 pi i k / W}  (gives W * x after the length-M inverse)
        for (int u = threadIdx.x; u < G * M; u += blockDim.x) {
            const int g = u % G, k = u / G;
            const float2 a = cur[g * Wh + k], b = cconj(cur[g * Wh + M - k]);
            const float2 e = cadd(a, b), o = cmul(csub(a, b), cconj(__ldg(twh + k)));
            Wk[at<G>(k, g)] = make_float2(e.x - o.y, e.y + o.x);
        }
        __syncthreads();
        const float2 *z = fft_any<MS, G, G, true, CT>(Wk, cur, p, tw);
        float fe = 0.f;
        for (int u = threadIdx.x; u < G * M; u += blockDim.x) {
            const int g = u % G, m = u / G, y = y0 + g;
            if (y >= H) continue;
            const float2 v = z[at<G>(m, g)];  // C(y, 2m), C(y, 2m + 1)
            const bool ynear = min(y, H - y) <= r;
            const int x0 = 2 * m, x1 = 2 * m + 1;
            if (!(ynear && min(x0, W - x0) <= r)) fe = __fmaf_rn(v.x, v.x, fe);
            if (!(ynear && min(x1, W - x1) <= r)) fe = __fmaf_rn(v.y, v.y, fe);
            const long long i0 = (long long)y * W + x0;
            if (v.x > bv || (v.x == bv && i0 < bi)) { bv = v.x; bi = i0; }
            if (v.y > bv || (v.y == bv && i0 + 1 < bi)) { bv = v.y; bi = i0 + 1; }
            if (y == 0 && m == 0) c0[q] = v.x;
        }
        acc += (double)fe;
        __syncthreads();  // Wk / cur are reused by the next iteration
    }
    cp_async_wait<0>();
    __syncthreads();
    // block reduction scratch in the now idle work buffer
    double *sh = reinterpret_cast<double *>(Wk);
    float *sv = reinterpret_cast<float *>(sh + 32);
    long long *si = reinterpret_cast<long long *>(sv + CT);
    const double e = block_sum_d(acc, sh);
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

// ---------------------------------------------------------------------------
// Warp-per-row forms of the two row passes for rows of 1920 samples (M = 960
// complex points, 960 = 32 x 30).  Lane n1 takes the 30-point DFT of
// z[n1 + 32 n2] (n2 = 0..29) in registers (radix 2 over two 15-point DFTs,
// those by the prime-factor map) and multiplies it by w_960^{n1 k2}; one
// transpose through the warp's own shared buffer; lane k2 (0..29) then takes
// the 32-point DFT (8 x 4) over n1, which gives Z[k2 + 30 k1].  A warp owns
// its row and synchronises only with itself: no block barrier, one shared-
// memory exchange per transform instead of three Stockham passes.
constexpr int RM = 960, RP = 32, RQ = 30;  // M = RP * RQ
constexpr int RTS = RP + 1;                 // transpose row stride (float2): at most 2-way conflicts
constexpr int RBUF = RQ * RTS;              // 990 float2 per warp (also holds the 960 results)

__device__ __forceinline__ float2 twm(const float2 *__restrict__ tw, int i) { return __ldg(tw + i); }  // w_960^i

// 30-point DFT (forward) of v[0..29] in place
__device__ __forceinline__ void dft30(float2 *v, const float2 *__restrict__ tw) {
    float2 e[15], o[15];
#pragma unroll
    for (int j = 0; j < 15; ++j) {
        e[j] = v[2 * j];
        o[j] = v[2 * j + 1];
    }
    Dft<15>::run(e);
    Dft<15>::run(o);
#pragma unroll
    for (int k = 0; k < 15; ++k) {
        const float2 t = k == 0 ? o[0] : cmul(o[k], twm(tw, 32 * k));  // w_30^k = w_960^{32 k}
        v[k] = cadd(e[k], t);
        v[k + 15] = csub(e[k], t);
    }
}

// 32-point DFT (forward) of u[0..31] in place: 8 x 4
__device__ __forceinline__ void dft32(float2 *u, const float2 *__restrict__ tw) {
    float2 t[8][4];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
#pragma unroll
        for (int j = 0; j < 4; ++j) t[b][j] = u[b + 8 * j];
        Dft<4>::run(t[b]);
#pragma unroll
        for (int k2 = 1; k2 < 4; ++k2)
            if (b) t[b][k2] = cmul(t[b][k2], twm(tw, 30 * b * k2));  // w_32^{b k2} = w_960^{30 b k2}
    }
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
        float2 sv[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) sv[b] = t[b][k2];
        Dft<8>::run(sv);
#pragma unroll
        for (int k1 = 0; k1 < 8; ++k1) u[k2 + 4 * k1] = sv[k1];
    }
}

// The 960-point transform of a warp's row, lane n1 holding v[n2] = z[n1 + 32 n2]
// (unnormalised; INV: exponent sign +1, as conj(DFT(conj z))); the result
// Z[0..959] is left in buf, visible to the whole warp.
template <bool INV>
__device__ __forceinline__ void fft960_warp(float2 *v, float2 *buf, const float2 *__restrict__ tw, int lane) {
    if (INV) {
#pragma unroll
        for (int n2 = 0; n2 < RQ; ++n2) v[n2] = cconj(v[n2]);
    }
    dft30(v, tw);
#pragma unroll
    for (int k2 = 0; k2 < RQ; ++k2) buf[k2 * RTS + lane] = (k2 && lane) ? cmul(v[k2], twm(tw, lane * k2)) : v[k2];
    __syncwarp();
    float2 u[RP];
    if (lane < RQ) {
#pragma unroll
        for (int n1 = 0; n1 < RP; ++n1) u[n1] = buf[lane * RTS + n1];
    }
    __syncwarp();
    if (lane < RQ) {
        dft32(u, tw);
#pragma unroll
        for (int k1 = 0; k1 < RP; ++k1) buf[lane + RQ * k1] = INV ? cconj(u[k1]) : u[k1];
    }
    __syncwarp();
}

// Forward row pass, rows of 2 * 960 real samples: half spectra of 961 bins
// (pitch ldo), each warp a row at a time.  Bounded to 128 registers (four
// blocks per SM; a few spilled values): 0.19 ms per video step against
// 0.27 ms at 168 registers and three blocks.
template <int NW>
__global__ void __launch_bounds__(32 * NW, 4) k_rfft_rows_w(const float *__restrict__ x, float2 *__restrict__ out,
                                                         long long nrows, int ldo, const float2 *__restrict__ twg) {
    __shared__ __align__(16) float2 sbuf[NW][RBUF];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2 *buf = sbuf[warp];
    const float2 *__restrict__ twh = twg + RM;  // w_1920^k, k <= 960
    for (long long r = (long long)blockIdx.x * NW + warp; r < nrows; r += (long long)gridDim.x * NW) {
        const float2 *z = reinterpret_cast<const float2 *>(x + r * (2 * RM));
        float2 v[RQ];
#pragma unroll
        for (int n2 = 0; n2 < RQ; ++n2) v[n2] = __ldg(z + lane + RP * n2);
        fft960_warp<false>(v, buf, twg, lane);
        // split step: X_k = (Z_k + conj Z_{M-k}) / 2 - i w_W^k (Z_k - conj Z_{M-k}) / 2
        for (int k = lane; k <= RM; k += 32) {
            const float2 zk = buf[k == RM ? 0 : k];
            const float2 zc = cconj(buf[k == 0 ? 0 : RM - k]);
            const float2 sm2 = cadd(zk, zc), wd = cmul(__ldg(twh + k), csub(zk, zc));
            if (PRNU_DCHECK(k < ldo, k)) out[r * ldo + k] = make_float2(0.5f * (sm2.x + wd.y), 0.5f * (sm2.y - wd.x));
        }
        __syncwarp();  // buf is rewritten by the warp's next row
    }
}

// Inverse row pass and PCE partials (as k_corr_rows), each warp a row at a
// time; three blocks per SM (168 registers, no spill: 0.15 ms per video step
// against 0.17 ms under the 128-register bound).
template <int NW>
__global__ void __launch_bounds__(32 * NW, 3) k_corr_rows_w(const float2 *__restrict__ Zall, int H, int W, int ld, int r,
                                                         const float2 *__restrict__ twg, double *part_e,
                                                         float *part_v, long long *part_i, float *c0) {
    __shared__ __align__(16) float2 sbuf[NW][RBUF];
    __shared__ double she[NW];
    __shared__ float shv[NW];
    __shared__ long long shi[NW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2 *buf = sbuf[warp];
    const int q = blockIdx.y;
    const float2 *Z = Zall + (long long)q * H * ld;
    const float2 *__restrict__ twh = twg + RM;
    double acc = 0.0;
    float bv = -__int_as_float(0x7f800000);
    long long bi = LLONG_MAX;
    for (int y = blockIdx.x * NW + warp; y < H; y += gridDim.x * NW) {
        const float2 *row = Z + (long long)y * ld;
        // split step: Z'_k = E_k + i O_k, E_k = X_k + conj X_{M-k},
        // O_k = (X_k - conj X_{M-k}) e^{+2 pi i k / W}  (gives W * x after the inverse)
        float2 v[RQ];
#pragma unroll
        for (int n2 = 0; n2 < RQ; ++n2) {
            const int k = lane + RP * n2;
            if (!PRNU_DCHECK(RM - k < ld, k)) continue;
            const float2 a = __ldg(row + k), b = cconj(__ldg(row + RM - k));
            const float2 e = cadd(a, b), o = cmul(csub(a, b), cconj(__ldg(twh + k)));
            v[n2] = make_float2(e.x - o.y, e.y + o.x);
        }
        fft960_warp<true>(v, buf, twg, lane);
        // energy outside the neighbourhood of zero shift (only the rows within r
        // of row 0 test columns), the row's first maximum in this lane, C(0, 0)
        float fe = 0.f, rv = -__int_as_float(0x7f800000);
        int rx = 0;
        const bool ynear = min(y, H - y) <= r;
        if (ynear) {
            for (int m = lane; m < RM; m += 32) {
                const float2 val = buf[m];  // C(y, 2m), C(y, 2m + 1)
                const int x0 = 2 * m, x1 = 2 * m + 1;
                if (min(x0, W - x0) > r) fe = __fmaf_rn(val.x, val.x, fe);
                if (min(x1, W - x1) > r) fe = __fmaf_rn(val.y, val.y, fe);
                if (val.x > rv) { rv = val.x; rx = x0; }
                if (val.y > rv) { rv = val.y; rx = x1; }
            }
        } else {
            for (int m = lane; m < RM; m += 32) {
                const float2 val = buf[m];
                fe = __fmaf_rn(val.x, val.x, fe);
                fe = __fmaf_rn(val.y, val.y, fe);
                if (val.x > rv) { rv = val.x; rx = 2 * m; }
                if (val.y > rv) { rv = val.y; rx = 2 * m + 1; }
            }
        }
        // rows come in increasing order per lane, so a tie keeps the earlier (smaller) index
        if (rv > bv) {
            bv = rv;
            bi = (long long)y * W + rx;
        }
        if (y == 0 && lane == 0) c0[q] = buf[0].x;
        acc += (double)fe;
        __syncwarp();  // buf is rewritten by the warp's next row
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_down_sync(0xffffffffu, acc, o);
        const float ov = __shfl_down_sync(0xffffffffu, bv, o);
        const long long oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) {
            bv = ov;
            bi = oi;
        }
    }
    if (lane == 0) {
        she[warp] = acc;
        shv[warp] = bv;
        shi[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double e = 0.0;
        float v0 = shv[0];
        long long i0 = shi[0];
        for (int w = 0; w < NW; ++w) {
            e += she[w];
            if (shv[w] > v0 || (shv[w] == v0 && shi[w] < i0)) {
                v0 = shv[w];
                i0 = shi[w];
            }
        }
        const long long o = (long long)q * gridDim.x + blockIdx.x;
        part_e[o] = e;
        part_v[o] = v0;
        part_i[o] = i0;
    }
}

constexpr int kRowWarps = 4;  // warps (rows in flight) per block of the warp-per-row passes

// Opts each kernel instance, once per device, into the largest dynamic shared
// memory the device allows next to its static shared memory (a host-side
// attribute; each launch still asks only for what it uses, checked against
// that limit).  Repeating it from another thread is harmless.
template <auto Kern>
cudaError_t smem_attr(size_t bytes) {
    static int limit[64] = {};  // per device: 0 unset, else limit + 1
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (limit[dev] == 0) {
        int optin = 0;
        cudaFuncAttributes fa{};
        cudaError_t e;
        if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
        if ((e = cudaFuncGetAttributes(&fa, Kern)) != cudaSuccess) return e;
        const int dyn = optin - (int)fa.sharedSizeBytes;
        if ((e = cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn)) != cudaSuccess) return e;
        limit[dev] = dyn + 1;
    }
    return bytes < (size_t)limit[dev] ? cudaSuccess : cudaErrorInvalidConfiguration;
}

int rows_per_block(int M) { return M <= 1024 ? 4 : 2; }
// the inverse row pass takes two rows per block, so that three of its blocks
// (80 registers, 256 threads) fit an SM's shared memory
constexpr int kInvRows = 2;
// twiddles (M) and three buffers of G padded rows
size_t rows_buf(int M, int G) { return (size_t)G * padded_len(M + 1); }
// (k_corr_rows reuses its work buffer as 3328 bytes of reduction scratch)
size_t rows_smem(int M, int G) {
    return std::max(((size_t)M + 3 * rows_buf(M, G)) * sizeof(float2), (size_t)M * sizeof(float2) + 3328);
}
size_t rows_smem(int M) { return rows_smem(M, rows_per_block(M)); }
size_t cols_smem(int H, int tc) { return ((size_t)H + 2 * 2 * tc * (size_t)padded_len(H)) * sizeof(float2); }
// widest column tile whose block still fits twice per SM, else once
int cols_tile(int H) {
    for (int tc : {4, 2, 1})
        if (cols_smem(H, tc) <= 113 * 1024) return tc;
    for (int tc : {4, 2, 1})
        if (cols_smem(H, tc) <= 220 * 1024) return tc;
    return 0;
}

}  // namespace

bool fft_steps(int L, FftSteps *p) {
    if (L < 2) return false;
    const StaticPlan sp = static_plan(L);
    if (sp.np <= 0) return false;
    FftSteps s{};
    s.L = L;
    for (int i = 0; i < sp.np; ++i) s.radix |= (unsigned long long)sp.r[i] << (4 * s.np++);
    *p = s;
    return true;
}

bool corr_fft_supported(int H, int W) {
    FftSteps a, b;
    if (W % 2 || W < 4 || H < 2) return false;
    if (!fft_steps(W / 2, &a) || !fft_steps(H, &b)) return false;
    return rows_smem(W / 2) <= 220 * 1024 && cols_tile(H) > 0;
}

size_t corr_twiddle_count(int H, int W) { return (size_t)(W / 2) * 2 + 1 + H; }
int corr_pitch(int W) { return (W / 2 + 1 + 3) / 4 * 4; }

namespace {
template <auto Kern, int NT = CT, typename... Args>
cudaError_t launch(dim3 grid, size_t smem, cudaStream_t st, Args... args) {
    cudaError_t e = smem_attr<Kern>(smem);
    if (e != cudaSuccess) return e;
    Kern<<<grid, NT, smem, st>>>(args...);
    return cudaGetLastError();
}
// lengths with compiled-in pass plans (1920 x 1080 frames); others run the
// same passes with run-time strides
constexpr int kStaticM = 960, kStaticH = 1080;
}  // namespace

cudaError_t launch_corr_fft(const float *XY, float2 *F, float2 *tw, int n, int H, int W, int r, int nb,
                            double *part_e, float *part_v, long long *part_i, float *c0, int sms, cudaStream_t st,
                            int stage) {
    const int M = W / 2, Wh = M + 1, ld = corr_pitch(W);
    FftSteps pm, ph;
    if (!fft_steps(M, &pm) || !fft_steps(H, &ph)) return cudaErrorInvalidValue;
    const int G = rows_per_block(M);
    const size_t rs = rows_smem(M);
    if (stage == 0) {
        const int nt = corr_twiddle_count(H, W);
        k_twiddles<<<(nt + 255) / 256, 256, 0, st>>>(tw, M, H);
        const long long nrows = 2LL * n * H;
        const dim3 grid((unsigned)std::min<long long>((nrows + G - 1) / G, (long long)sms * (rs <= 113 * 1024 ? 2 : 1)));
        if (M == RM) {
            const dim3 gw((unsigned)std::min<long long>((nrows + kRowWarps - 1) / kRowWarps, (long long)sms * 8));
            k_rfft_rows_w<kRowWarps><<<gw, 32 * kRowWarps, 0, st>>>(XY, F, nrows, ld, (const float2 *)tw);
            return cudaGetLastError();
        }
        if (M == kStaticM)
            return launch<k_rfft_rows<4, kStaticM, CTW>, CTW>(grid, rs, st, XY, F, nrows, W, ld, pm, (const float2 *)tw);
        if (G == 4) return launch<k_rfft_rows<4, 0, CTW>, CTW>(grid, rs, st, XY, F, nrows, W, ld, pm, (const float2 *)tw);
        return launch<k_rfft_rows<2, 0, CTW>, CTW>(grid, rs, st, XY, F, nrows, W, ld, pm, (const float2 *)tw);
    }
    if (stage == 1) {
        const int tc = cols_tile(H);
        const size_t cs = cols_smem(H, tc);
        const dim3 grid((Wh + tc - 1) / tc, n);
        const float2 *twc = tw + 2 * M + 1;
        if (H == K4_L) {  // four-step form, K4_COLS columns per block
            const size_t s4 = (size_t)3 * K4_N2 * K4_SS * sizeof(float2);
            const dim3 g4((Wh + K4_COLS - 1) / K4_COLS, n);
            return launch<k_corr_columns_4s, K4_NT>(g4, s4, st, F, n, Wh, ld, twc);
        }
        if (H == kStaticH && tc == 2)
            return launch<k_corr_columns<2, kStaticH, CTH>, CTH>(grid, cs, st, F, n, H, Wh, ld, ph, twc);
        if (tc == 4) return launch<k_corr_columns<4, 0, CTW>, CTW>(grid, cs, st, F, n, H, Wh, ld, ph, twc);
        if (tc == 2) return launch<k_corr_columns<2, 0, CTW>, CTW>(grid, cs, st, F, n, H, Wh, ld, ph, twc);
        return launch<k_corr_columns<1, 0, CTW>, CTW>(grid, cs, st, F, n, H, Wh, ld, ph, twc);
    }
    const dim3 grid((unsigned)corr_rows_blocks(H, W, nb), n);
    const size_t ri = rows_smem(M, kInvRows);
    const float2 *Fc = F, *twc = tw;
    if (M == RM) {
        k_corr_rows_w<kRowWarps><<<grid, 32 * kRowWarps, 0, st>>>(Fc, H, W, ld, r, twc, part_e, part_v, part_i, c0);
        return cudaGetLastError();
    }
    if (M == kStaticM)
        return launch<k_corr_rows<kInvRows, kStaticM>>(grid, ri, st, Fc, H, W, ld, r, pm, twc, part_e, part_v, part_i,
                                                        c0);
    return launch<k_corr_rows<kInvRows, 0>>(grid, ri, st, Fc, H, W, ld, r, pm, twc, part_e, part_v, part_i, c0);
}

int corr_rows_blocks(int H, int W, int nb) {
    const int rows = W / 2 == RM ? kRowWarps : kInvRows;  // rows per block iteration
    return std::min(nb, (H + rows - 1) / rows);
}

}  // namespace prnu
