// k_shrink.cu -- local-variance Wiener shrink of detail coefficients (the
// denoiser of Mihcak et al., cited in Sec. IV-A and Sec. V; parameters are the
// build's reading).  For each coefficient c of a subband and each window w:
//   mean_w = (1/w^2) sum of c^2 over the w x w window (periodic wrap),
//   var = max(0, min_w mean_w - s0^2),   noise = c s0^2 / (var + s0^2)
// (0 when var + s0^2 == 0, which forces c == 0).
//
// A 32 x 32 output tile stages c^2 with a 4-sample halo in shared memory; the
// box sums are separable: per-window row sums, then column sums.
#include "kernels.cuh"

namespace prnu {

constexpr int ST = 32, SH = kMaxRadius, SE = ST + 2 * SH;  // tile, halo, extended tile

__global__ void __launch_bounds__(256) k_shrink(ShrinkArgs a) {
    __shared__ float c2[SE][SE + 1];
    __shared__ float rs[4][SE][ST + 1];
    const int plane = blockIdx.z;
    const int y0 = blockIdx.y * ST, x0 = blockIdx.x * ST;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const float *in = a.in + (long long)plane * a.R * a.Cc;

    for (int i = tid; i < SE * SE; i += 256) {
        const int r = i / SE, c = i - r * SE;
        const int gy = wrap(y0 + r - SH, a.R), gx = wrap(x0 + c - SH, a.Cc);
        const float v = __ldg(in + (long long)gy * a.Cc + gx);
        c2[r][c] = v * v;
    }
    __syncthreads();

    for (int i = tid; i < SE * ST; i += 256) {
        const int r = i / ST, x = i - r * ST;
        for (int w = 0; w < a.win.n; ++w) {
            const int rad = a.win.r[w];
            float s = 0.f;
            for (int dx = -rad; dx <= rad; ++dx) s += c2[r][x + SH + dx];
            rs[w][r][x] = s;
        }
    }
    __syncthreads();

    const int x = threadIdx.x;
    for (int yl = threadIdx.y; yl < ST; yl += blockDim.y) {
        const int gy = y0 + yl, gx = x0 + x;
        if (gy >= a.R || gx >= a.Cc) continue;
        float vmin = __int_as_float(0x7f800000);  // +inf
        for (int w = 0; w < a.win.n; ++w) {
            const int rad = a.win.r[w];
            float s = 0.f;
            for (int dy = -rad; dy <= rad; ++dy) s += rs[w][yl + SH + dy][x];
            vmin = fminf(vmin, s * a.win.inv[w]);
        }
        const float c = in[(long long)gy * a.Cc + gx];
        const float s2 = a.s2_dev ? (float)a.s2_dev[1] : a.s2;
        const float var = fmaxf(0.f, vmin - s2);
        const float den = var + s2;
        a.out[(long long)plane * a.R * a.Cc + (long long)gy * a.Cc + gx] = den > 0.f ? __fdiv_rn(c * s2, den) : 0.f;
    }
}

cudaError_t launch_shrink(const ShrinkArgs &a, cudaStream_t st) {
    dim3 block(32, 8);
    dim3 grid((unsigned)((a.Cc + ST - 1) / ST), (unsigned)((a.R + ST - 1) / ST), (unsigned)a.nplanes);
    k_shrink<<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace prnu
