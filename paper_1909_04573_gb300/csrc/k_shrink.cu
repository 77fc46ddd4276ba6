// k_shrink.cu -- local-variance Wiener shrink of detail coefficients (the
// denoiser of Mihcak et al., cited in Sec. III-A and Sec. IV; parameters are the
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


// ---------------------------------------------------------------------------
// Packed variant for the standard windows {3, 5, 7, 9} on subbands whose width
// is a multiple of 4.  Same arithmetic per coefficient (direct sums of c^2,
// nested in the row direction), issued as float32x2 operations: a thread's
// values come in pairs of adjacent columns, so every shared-memory load of
// the box sums is an aligned 64-bit load and every add a packed add.
//   staging: the extended tile (40 x 40) of c^2 is loaded as 4-wide groups
//            (periodic wrap per group) and kept twice, as is and shifted left
//            by one column, so the pair starting at any column is aligned;
//   rows:    an item is one extended row and 4 output columns: 11 pair loads
//            give the nested row sums of radii 1..4 for both column pairs;
//   columns: a thread owns 2 output rows x 2 columns; per radius the two rows
//            share the 2d middle terms of their column sums.
using f2 = unsigned long long;  // two float32 in one 64-bit register

__device__ __forceinline__ f2 pk2(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void up2(f2 v, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 lds2(const float *p) { return *reinterpret_cast<const f2 *>(p); }

template <class T> struct Vec4;
template <> struct Vec4<float> {
    __device__ static float4 ld(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
};
template <> struct Vec4<__half> {
    __device__ static float4 ld(const __half *p) {
        const uint2 u = __ldg(reinterpret_cast<const uint2 *>(p));
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
};
template <> struct Vec4<__nv_bfloat16> {
    __device__ static float4 ld(const __nv_bfloat16 *p) {
        const uint2 u = __ldg(reinterpret_cast<const uint2 *>(p));
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
};

constexpr int XS = 42;  // row stride of the staged c^2 (even: 8-byte pairs; 2 mod 4: no bank overlap of rows)

template <bool S2DEV, class T>
__global__ void __launch_bounds__(256) k_shrink_x2(ShrinkArgs a) {
    __shared__ __align__(16) float c2[SE][XS];   // c^2, extended columns 0..39
    __shared__ __align__(16) float c2s[SE][XS];  // c2s[r][k] = c2[r][k + 1]
    __shared__ __align__(16) float rs[4][SE][ST];
    const int plane = blockIdx.z;
    const int y0 = blockIdx.y * ST, x0 = blockIdx.x * ST;
    const int tid = threadIdx.x;
    const T *in = static_cast<const T *>(a.in) + (long long)plane * a.R * a.Cc;
    T *out = static_cast<T *>(a.out) + (long long)plane * a.R * a.Cc;

    // staging: 40 rows x 10 groups of 4 columns, both loads of a thread first
    const int nq = a.Cc >> 2;
    constexpr int NI = SE * (SE / 4);  // 400 groups: items tid and tid + 256
    float4 v[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int it = tid + 256 * k;
        if (it < NI) {
            const int r = it / (SE / 4), j = it - r * (SE / 4);
            v[k] = Vec4<T>::ld(in + (long long)wrap_near(y0 + r - SH, a.R) * a.Cc +
                               4 * wrap_near((x0 >> 2) - 1 + j, nq));
        }
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int it = tid + 256 * k;
        if (it < NI) {
            const int r = it / (SE / 4), j = it - r * (SE / 4);
            const float q0 = v[k].x * v[k].x, q1 = v[k].y * v[k].y, q2 = v[k].z * v[k].z, q3 = v[k].w * v[k].w;
            *reinterpret_cast<float2 *>(&c2[r][4 * j]) = make_float2(q0, q1);
            *reinterpret_cast<float2 *>(&c2[r][4 * j + 2]) = make_float2(q2, q3);
            if (j > 0) c2s[r][4 * j - 1] = q0;
            *reinterpret_cast<float2 *>(&c2s[r][4 * j]) = make_float2(q1, q2);
            c2s[r][4 * j + 2] = q3;
        }
    }
    __syncthreads();

    // rows: item = (extended row r, output columns 4g .. 4g+3)
    for (int it = tid; it < SE * (ST / 4); it += 256) {
        const int r = it >> 3, g = it & 7;
        const int xc = 4 * g + SH;  // extended column of output column 4g
        // P[i + 4] = (c2[xc + i], c2[xc + i + 1]), i = -4 .. 6
        f2 P[11];
#pragma unroll
        for (int i = -4; i <= 6; ++i)
            P[i + 4] = (i & 1) ? lds2(&c2s[r][xc + i - 1]) : lds2(&c2[r][xc + i]);
        f2 s = add2(P[4], add2(P[3], P[5]));  // columns (4g, 4g+1)
        f2 t = add2(P[6], add2(P[5], P[7]));  // columns (4g+2, 4g+3)
#pragma unroll
        for (int d = 1; d <= 4; ++d) {
            if (d > 1) {
                s = add2(s, add2(P[4 - d], P[4 + d]));
                t = add2(t, add2(P[6 - d], P[6 + d]));
            }
            float s0, s1, t0, t1;
            up2(s, s0, s1);
            up2(t, t0, t1);
            *reinterpret_cast<float4 *>(&rs[d - 1][r][4 * g]) = make_float4(s0, s1, t0, t1);
        }
    }
    __syncthreads();

    // columns: thread = (column pair p, row pair rp); its coefficients are
    // loaded first so the loads overlap the sums
    const int p = tid & 15, rp = tid >> 4;
    const int yb = 2 * rp;  // output rows yb, yb+1
    const int gx = x0 + 2 * p;
    float cv[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int gy = y0 + yb + k;
        if (gy < a.R && gx < a.Cc) {
            cv[2 * k] = ldf<T>(in + (long long)gy * a.Cc + gx);
            cv[2 * k + 1] = ldf<T>(in + (long long)gy * a.Cc + gx + 1);
        }
    }
    f2 m0 = pk2(__int_as_float(0x7f800000), __int_as_float(0x7f800000)), m1 = m0;
#pragma unroll
    for (int d = 1; d <= 4; ++d) {
        // rows yb - d .. yb + 1 + d of rs (extended row = output row + SH)
        f2 core = lds2(&rs[d - 1][yb + SH - d + 1][2 * p]);
#pragma unroll
        for (int j = 2 - d; j <= d; ++j) core = add2(core, lds2(&rs[d - 1][yb + SH + j][2 * p]));
        const f2 b0 = add2(lds2(&rs[d - 1][yb + SH - d][2 * p]), core);
        const f2 b1 = add2(core, lds2(&rs[d - 1][yb + SH + d + 1][2 * p]));
        const f2 iw = pk2(a.win.inv[d - 1], a.win.inv[d - 1]);
        const f2 v0 = mul2(b0, iw), v1 = mul2(b1, iw);
        float u0, u1, w0, w1, n0, n1, o0, o1;
        up2(v0, u0, u1);
        up2(v1, w0, w1);
        up2(m0, n0, n1);
        up2(m1, o0, o1);
        m0 = pk2(fminf(n0, u0), fminf(n1, u1));
        m1 = pk2(fminf(o0, w0), fminf(o1, w1));
    }
    const float s2 = S2DEV ? (float)a.s2_dev[1] : a.s2;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int gy = y0 + yb + k;
        if (gy >= a.R || gx >= a.Cc) continue;
        float mA, mB;
        up2(k ? m1 : m0, mA, mB);
        T *dst = out + (long long)gy * a.Cc + gx;
        const float denA = fmaxf(0.f, mA - s2) + s2, denB = fmaxf(0.f, mB - s2) + s2;
        stf<T>(dst, denA > 0.f ? __fdividef(cv[2 * k] * s2, denA) : 0.f);
        stf<T>(dst + 1, denB > 0.f ? __fdividef(cv[2 * k + 1] * s2, denB) : 0.f);
    }
}

template <class T>
static void launch_shrink_t(const ShrinkArgs &a, cudaStream_t st) {
    dim3 block(32, 8);
    dim3 grid((unsigned)((a.Cc + ST - 1) / ST), (unsigned)((a.R + ST - 1) / ST), (unsigned)a.nplanes);
    const bool std4 = a.win.n == 4 && a.win.r[0] == 1 && a.win.r[1] == 2 && a.win.r[2] == 3 && a.win.r[3] == 4;
    if (std4 && a.Cc % 4 == 0) {  // packed path (aligned 4-wide groups)
        if (a.s2_dev)
            k_shrink_x2<true, T><<<grid, 256, 0, st>>>(a);
        else
            k_shrink_x2<false, T><<<grid, 256, 0, st>>>(a);
    } else if (std4 && !a.s2_dev)
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
