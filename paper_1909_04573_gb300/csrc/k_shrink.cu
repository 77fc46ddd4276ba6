// k_shrink.cu -- local-variance Wiener shrink of detail coefficients (the
// denoiser of Mihcak et al., cited in Sec. III-A and Sec. IV; parameters are the
// build's reading).  For each coefficient c of a subband and each window w:
//   mean_w = (1/w^2) sum of c^2 over the w x w window (periodic wrap),
//   var = max(0, min_w mean_w - s0^2),   noise = c s0^2 / (var + s0^2)
// (0 when var + s0^2 == 0, which forces c == 0).
//
// The box sums are separable: per-window row sums, then column sums.  The
// standard windows on widths that are multiples of 4 take k_shrink_strip
// (register column sums down a strip); other window sets and widths take
// k_shrink (a 32 x 32 tile with both sums through shared memory).
#include <type_traits>

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
            if (c < SE && PRNU_DCHECK(srcx[k] >= 0 && srcx[k] < a.Cc && rowoff < (long long)a.R * a.Cc, srcx[k])) {
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
// float32x2 helpers: two adjacent columns' values in one 64-bit register,
// added and multiplied with the packed Blackwell instructions.
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

// ---------------------------------------------------------------------------
// Standard windows {3, 5, 7, 9} on subbands whose width is a multiple of 4.
// A block covers 64 columns x SS_H rows; each thread owns two adjacent
// columns and walks down a strip of SS_SL rows of the coefficients staged
// with a 4-sample periodic halo.  Per staged row, five aligned pair loads
// give c at columns x-4 .. x+5, and packed float32x2 operations form c^2 and
// the nested row sums of radii 1..4; the box sum of radius d is a direct sum
// of the last 2d+1 rows' row sums, kept in registers, and two consecutive
// output rows share their 2d middle terms.  No row-sum array goes through
// shared memory.
constexpr int SS_W = 64, SS_WARPS = 4, SS_SL = 34;  // 544 = 4 x 136: level-1 subbands of 1088-row frames
static_assert(SS_SL % 2 == 0, "output rows come in pairs");
constexpr int SS_H = SS_WARPS * SS_SL;
constexpr int SS_XS = SS_W + 2 * SH;  // 72 staged columns (float4-aligned rows)

__device__ __forceinline__ void cp_async16(float *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// float32 subbands (WS): each warp stages its own strip (SS_SL + 8 rows) with
// cp.async in three row groups and starts on the first while the others are
// in flight -- no block barrier; 16-bit subbands share one converted tile.
template <bool S2DEV, class T>
__global__ void __launch_bounds__(32 * SS_WARPS) k_shrink_strip(ShrinkArgs a) {
    constexpr bool WS = std::is_same<T, float>::value;
    constexpr int SR = SS_SL + 2 * SH, GPR = SS_XS / 4;  // staged rows per strip, 4-column groups per row
    __shared__ __align__(16) float cs[WS ? SS_WARPS * SR * SS_XS : (SS_H + 2 * SH) * SS_XS];
    const int plane = blockIdx.z;
    const int y0 = blockIdx.y * SS_H, x0 = blockIdx.x * SS_W;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const T *in = static_cast<const T *>(a.in) + (long long)plane * a.R * a.Cc;
    T *out = static_cast<T *>(a.out) + (long long)plane * a.R * a.Cc;
    const int nq = a.Cc >> 2;
    const int ys = y0 + warp * SS_SL;  // first output row of this warp's strip

    if constexpr (!WS) {
        // staging: (SS_H + 8) rows x 18 groups of 4 columns (periodic wrap per group)
        constexpr int NG = (SS_H + 2 * SH) * GPR;
#pragma unroll 4
        for (int it = tid; it < NG; it += 32 * SS_WARPS) {
            const int r = it / GPR, j = it - r * GPR;
            const float4 v = Vec4<T>::ld(in + (long long)wrap_near(y0 + r - SH, a.R) * a.Cc +
                                         4 * wrap_near((x0 >> 2) - 1 + j, nq));
            *reinterpret_cast<float4 *>(&cs[r * SS_XS + 4 * j]) = v;
        }
        __syncthreads();
    }
    if (ys >= a.R) return;  // whole strip past the plane (no barrier follows)
    float *const wsm = WS ? cs + warp * SR * SS_XS : cs + warp * SS_SL * SS_XS;
    if constexpr (WS) {
        static_assert(SR % 3 == 0, "three equal row groups");
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            for (int it = lane; it < (SR / 3) * GPR; it += 32) {
                const int r = g * (SR / 3) + it / GPR, j = it % GPR;
                if (!PRNU_DCHECK(4 * wrap_near((x0 >> 2) - 1 + j, nq) + 3 < a.Cc, j)) continue;
                cp_async16(wsm + r * SS_XS + 4 * j, in + (long long)wrap_near(ys - SH + r, a.R) * a.Cc +
                                                        4 * wrap_near((x0 >> 2) - 1 + j, nq));
            }
            cp_async_commit();
        }
    }
    const int gx = x0 + 2 * lane;
    const float s2 = S2DEV ? (float)a.s2_dev[1] : a.s2;
    const f2 iw1 = pk2(a.win.inv[0], a.win.inv[0]), iw2 = pk2(a.win.inv[1], a.win.inv[1]);
    const f2 iw3 = pk2(a.win.inv[2], a.win.inv[2]), iw4 = pk2(a.win.inv[3], a.win.inv[3]);
    // staged row of strip row i: wsm + i * SS_XS; lane's pairs start at column 2 lane
    const float *base = wsm + 2 * lane;
    f2 R1[SS_SL + 8], R2[SS_SL + 8], R3[SS_SL + 8], R4[SS_SL + 8];
#pragma unroll
    for (int i = 0; i < SS_SL + 8; ++i) {
        if constexpr (WS) {  // row group i / 14 has landed (each lane waits for its copies, then the warp syncs)
            if (i == 0) cp_async_wait<2>();
            if (i == SR / 3) cp_async_wait<1>();
            if (i == 2 * SR / 3) cp_async_wait<0>();
            if (i == 0 || i == SR / 3 || i == 2 * SR / 3) __syncwarp();
        }
        const float *row = base + i * SS_XS;
        const f2 e0 = lds2(row), e1 = lds2(row + 2), e2 = lds2(row + 4), e3 = lds2(row + 6), e4 = lds2(row + 8);
        const f2 q0 = mul2(e0, e0), q1 = mul2(e1, e1), q2 = mul2(e2, e2), q3 = mul2(e3, e3), q4 = mul2(e4, e4);
        float a0, a1, b0, b1, c0, c1, d0, d1, g0, g1;
        up2(q0, a0, a1);
        up2(q1, b0, b1);
        up2(q2, c0, c1);
        up2(q3, d0, d1);
        up2(q4, g0, g1);
        // columns (x, x+1): q_k = c^2 at (x-4+2k, x-3+2k); odd pairs straddle them
        const f2 om3 = pk2(a1, b0), om1 = pk2(b1, c0), op1 = pk2(c1, d0), op3 = pk2(d1, g0);
        R1[i] = add2(q2, add2(om1, op1));
        R2[i] = add2(R1[i], add2(q1, q3));
        R3[i] = add2(R2[i], add2(om3, op3));
        R4[i] = add2(R3[i], add2(q0, q4));
        // output rows in pairs (o, o+1), o = i - 9 even: their box sums of
        // radius d share the 2d middle row sums (direct sums of the same terms)
        if (i >= 9 && ((i - 9) & 1) == 0) {
            const int o = i - 9, c = i - 5;  // first output row of the pair, its staged row (strip-relative)
            f2 m1 = R1[c], m2 = R2[c - 1], m3 = R3[c - 2], m4 = R4[c - 3];
            m1 = add2(m1, R1[c + 1]);
#pragma unroll
            for (int j = 0; j < 3; ++j) m2 = add2(m2, R2[c + j]);
#pragma unroll
            for (int j = -1; j < 4; ++j) m3 = add2(m3, R3[c + j]);
#pragma unroll
            for (int j = -2; j < 5; ++j) m4 = add2(m4, R4[c + j]);
            const f2 b[2][4] = {{add2(R1[c - 1], m1), add2(R2[c - 2], m2), add2(R3[c - 3], m3), add2(R4[c - 4], m4)},
                                {add2(m1, R1[c + 2]), add2(m2, R2[c + 3]), add2(m3, R3[c + 4]), add2(m4, R4[c + 5])}};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float m1a, m1b, m2a, m2b, m3a, m3b, m4a, m4b;
                up2(mul2(b[h][0], iw1), m1a, m1b);
                up2(mul2(b[h][1], iw2), m2a, m2b);
                up2(mul2(b[h][2], iw3), m3a, m3b);
                up2(mul2(b[h][3], iw4), m4a, m4b);
                const float mA = fminf(fminf(m1a, m2a), fminf(m3a, m4a));
                const float mB = fminf(fminf(m1b, m2b), fminf(m3b, m4b));
                const int gy = ys + o + h;
                if (gy < a.R && gx < a.Cc && PRNU_DCHECK(gx + 1 < a.Cc, gx)) {
                    float cA, cB;
                    up2(lds2(base + (c + h) * SS_XS + 4), cA, cB);
                    const float denA = fmaxf(0.f, mA - s2) + s2, denB = fmaxf(0.f, mB - s2) + s2;
                    T *dst = out + (long long)gy * a.Cc + gx;
                    stf<T>(dst, denA > 0.f ? __fdividef(cA * s2, denA) : 0.f);
                    stf<T>(dst + 1, denB > 0.f ? __fdividef(cB * s2, denB) : 0.f);
                }
            }
        }
    }
}

template <class T>
static void launch_shrink_t(const ShrinkArgs &a, cudaStream_t st, int choice) {
    dim3 block(32, 8);
    dim3 grid((unsigned)((a.Cc + ST - 1) / ST), (unsigned)((a.R + ST - 1) / ST), (unsigned)a.nplanes);
    const bool std4 = a.win.n == 4 && a.win.r[0] == 1 && a.win.r[1] == 2 && a.win.r[2] == 3 && a.win.r[3] == 4;
    if (std4 && a.Cc % 4 == 0 && choice == 0) {  // strip path (aligned 4-wide groups)
        dim3 g2((unsigned)((a.Cc + SS_W - 1) / SS_W), (unsigned)((a.R + SS_H - 1) / SS_H), (unsigned)a.nplanes);
        if (a.s2_dev)
            k_shrink_strip<true, T><<<g2, 32 * SS_WARPS, 0, st>>>(a);
        else
            k_shrink_strip<false, T><<<g2, 32 * SS_WARPS, 0, st>>>(a);
    } else if (std4 && !a.s2_dev)
        k_shrink<true, false, T><<<grid, block, 0, st>>>(a);
    else if (std4)
        k_shrink<true, true, T><<<grid, block, 0, st>>>(a);
    else if (!a.s2_dev)
        k_shrink<false, false, T><<<grid, block, 0, st>>>(a);
    else
        k_shrink<false, true, T><<<grid, block, 0, st>>>(a);
}

cudaError_t launch_shrink(const ShrinkArgs &a, cudaStream_t st, int choice) {
    if (a.sdt == SB_F16)
        launch_shrink_t<__half>(a, st, choice);
    else if (a.sdt == SB_BF16)
        launch_shrink_t<__nv_bfloat16>(a, st, choice);
    else
        launch_shrink_t<float>(a, st, choice);
    return cudaGetLastError();
}

}  // namespace prnu
