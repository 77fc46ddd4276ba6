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
constexpr int C2S = SE + 4;                                 // c^2 row stride (float4-aligned)

// STD: the windows are exactly {3, 5, 7, 9} (radii 1..4).  Register-blocked:
// a row-sum item covers 4 consecutive columns of one extended row (12 c^2
// values in, 4 x 4 nested sums out) and a column-sum item covers 4 consecutive
// output rows of one column (the 12 row sums of each radius it needs are read
// once).  Every window sum is a direct sum of its terms (no running
// subtraction, so a large coefficient leaving a window cannot cancel the small
// ones).  Other window sets take the generic path.  S2DEV: sigma0^2 is read
// from device memory (the DFT-domain Wiener filter, whose noise variance is
// computed on the device).
template <bool STD, bool S2DEV, class T>
__global__ void __launch_bounds__(256) k_shrink(ShrinkArgs a) {
    __shared__ __align__(16) float c2[SE][C2S];
    __shared__ float rs[4][SE][ST + 1];
    const int plane = blockIdx.z;
    const int y0 = blockIdx.y * ST, x0 = blockIdx.x * ST;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * 32 + tx;
    const T *in = static_cast<const T *>(a.in) + (long long)plane * a.R * a.Cc;
    T *out = static_cast<T *>(a.out) + (long long)plane * a.R * a.Cc;

    int srcx[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) srcx[k] = wrap_near(x0 + tx + 32 * k - SH, a.Cc);
    for (int r = ty; r < SE; r += 8) {
        const long long rowoff = (long long)wrap_near(y0 + r - SH, a.R) * a.Cc;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int c = tx + 32 * k;
            if (c < SE) {
                const float v = ldf<T>(in + rowoff + srcx[k]);
                c2[r][c] = v * v;
            }
        }
    }
    __syncthreads();

    if (STD) {
        // row sums: item = (extended row r, column group g of 4)
        for (int it = tid; it < SE * (ST / 4); it += 256) {
            const int r = it >> 3, g = it & 7;
            const float4 *row = reinterpret_cast<const float4 *>(&c2[r][0]);
            float v[12];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float4 t = row[g + k];
                v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {  // output column 4g+j sits at v[j+4]
                float s = v[j + 4];
#pragma unroll
                for (int d = 1; d <= 4; ++d) {
                    s += v[j + 4 - d] + v[j + 4 + d];
                    rs[d - 1][r][4 * g + j] = s;
                }
            }
        }
    } else {
        for (int r = ty; r < SE; r += 8) {
            const int x = tx + SH;
            for (int w = 0; w < a.win.n; ++w) {
                const int rad = a.win.r[w];
                float s = 0.f;
                for (int dx = -rad; dx <= rad; ++dx) s += c2[r][x + dx];
                rs[w][r][tx] = s;
            }
        }
    }
    __syncthreads();

    const float s2 = S2DEV ? (float)a.s2_dev[1] : a.s2;
    const int gx = x0 + tx;
    if (STD) {
        // column sums: thread (tx, ty) owns output rows 4ty .. 4ty+3
        const int yb = 4 * ty;
        float m[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) m[k] = __int_as_float(0x7f800000);
#pragma unroll
        for (int d = 1; d <= 4; ++d) {
            float col[12];
#pragma unroll
            for (int k = 0; k < 4 + 2 * d; ++k) col[k] = rs[d - 1][yb + SH - d + k][tx];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float s = 0.f;
#pragma unroll
                for (int j = 0; j <= 2 * d; ++j) s += col[k + j];
                m[k] = fminf(m[k], s * a.win.inv[d - 1]);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int gy = y0 + yb + k;
            if (gy >= a.R || gx >= a.Cc) continue;
            const float c = ldf<T>(in + (long long)gy * a.Cc + gx);
            const float var = fmaxf(0.f, m[k] - s2);
            const float den = var + s2;
            stf<T>(out + (long long)gy * a.Cc + gx, den > 0.f ? __fdividef(c * s2, den) : 0.f);
        }
    } else {
        for (int yl = ty; yl < ST; yl += 8) {
            const int gy = y0 + yl;
            if (gy >= a.R || gx >= a.Cc) continue;
            const int yc = yl + SH;
            float vmin = __int_as_float(0x7f800000);  // +inf
            for (int w = 0; w < a.win.n; ++w) {
                const int rad = a.win.r[w];
                float s = 0.f;
                for (int dy = -rad; dy <= rad; ++dy) s += rs[w][yc + dy][tx];
                vmin = fminf(vmin, s * a.win.inv[w]);
            }
            const float c = ldf<T>(in + (long long)gy * a.Cc + gx);
            const float var = fmaxf(0.f, vmin - s2);
            const float den = var + s2;
            stf<T>(out + (long long)gy * a.Cc + gx, den > 0.f ? __fdividef(c * s2, den) : 0.f);
        }
    }
}

template <class T>
static void launch_shrink_t(const ShrinkArgs &a, cudaStream_t st) {
    dim3 block(32, 8);
    dim3 grid((unsigned)((a.Cc + ST - 1) / ST), (unsigned)((a.R + ST - 1) / ST), (unsigned)a.nplanes);
    const bool std4 = a.win.n == 4 && a.win.r[0] == 1 && a.win.r[1] == 2 && a.win.r[2] == 3 && a.win.r[3] == 4;
    if (std4 && !a.s2_dev)
        k_shrink<true, false, T><<<grid, block, 0, st>>>(a);
    else if (std4)
        k_shrink<true, true, T><<<grid, block, 0, st>>>(a);
    else if (!a.s2_dev)
        k_shrink<false, false, T><<<grid, block, 0, st>>>(a);
    else
        k_shrink<false, true, T><<<grid, block, 0, st>>>(a);
}

cudaError_t launch_shrink(const ShrinkArgs &a, cudaStream_t st) {
    if (a.sdt == SB_F16)
        launch_shrink_t<__half>(a, st);
    else if (a.sdt == SB_BF16)
        launch_shrink_t<__nv_bfloat16>(a, st);
    else
        launch_shrink_t<float>(a, st);
    return cudaGetLastError();
}

}  // namespace prnu
