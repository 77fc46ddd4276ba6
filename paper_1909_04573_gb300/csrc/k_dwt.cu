// k_dwt.cu -- one level of the periodised orthonormal 2-D DWT (analysis),
// rows first then columns: a[n] = sum_k h[k] x[(2n+k) mod N],
// d[n] = sum_k g[k] x[(2n+k) mod N], g[k] = (-1)^k h[7-k].
//
// Difference form.  Input values are 128-ish pixel sums, the detail outputs
// are O(1) noise, so a plain float32 filter loses the result in the rounding
// of its large partial sums.  Every output instead works on differences to one
// reference sample of its own support, using sum_k g[k] = 0 and
// sum_k h[k] = sqrt(2) exactly:
//   row pass at (y, q), ref r = v[y][2q], delta_k = v[y][2q+k] - r:
//       lo = sqrt2 r + s,  s = sum_{k>=1} h[k] delta_k;   hi = t = sum g[k] delta_k
//   column pass at (p, q), rows y_j = 2p+j, D_j = r_{y_j} - r_{y_0}:
//       LL = 2 r_{y_0} + sqrt2 sum h_j D_j + sum h_j s_{y_j}
//       LH = sqrt2 sum g_j D_j + sum g_j s_{y_j}
//       HL = sum h_j t_{y_j},   HH = sum g_j t_{y_j}
// The large term 2 r appears only in LL, which is carried to the next level
// as an unevaluated float-float pair (hi, lo).  At level 1 the inputs are
// exact integer group sums (or float32 images), so the differences are exact.
// Details are scaled by 1/count (pixel units) when written; the LL chain stays
// in sum units.
//
// Two launch shapes: level 1 (the full-resolution planes) streams down strips
// with the row pass held in registers; levels >= 2 (a quarter of the samples
// or fewer, too few strips to keep the GPU busy) use shared-memory tiles.
#include "dwt_rows.cuh"

namespace prnu {

// Streaming layout: a warp owns 32 consecutive output columns q and a strip
// of SP output rows; each lane walks down its column.  The row pass of an
// input row y (ref, s, t) goes into a ring of the last 8 input rows held in
// registers; every two new input rows complete one output row (rows
// 2p..2p+7).  The ring slot of input row y is (y - 2p0) mod 8, so an unrolled
// body of 4 output rows uses fixed slots.  At level 1 the interior warps read
// their input rows from a per-warp shared-memory ring that cp.async fills
// ahead of use (below); the mirrored edge warps, and levels above 1, read
// global memory through L1 (four float2 per row where aligned).  No block
// barriers: each warp synchronises only with itself.
// Launch shapes (output rows per strip SP, a multiple of 4, and warps per
// block side by side in q) are template parameters; prnu_autotune picks one
// per geometry among kStreamShapes.

struct RowIn {
    const float *h, *l;       // row base of the high / low parts (l unused at level 1)
};

template <bool LEVEL1>
struct Lane {
    int col[8];               // source column of input samples 2q..2q+7
    bool fast;                // warp-uniform: columns are 2q..2q+7 directly, float2-aligned
};

// raw samples 2q..2q+7 of one input row (high and, above level 1, low parts)
template <bool LEVEL1>
__device__ __forceinline__ void row_load(const RowIn &row, const Lane<LEVEL1> &L, int q2, float *v, float *w) {
    if (L.fast) {
        const float2 *ph = reinterpret_cast<const float2 *>(row.h + q2);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 u = __ldg(ph + j);
            v[2 * j] = u.x;
            v[2 * j + 1] = u.y;
        }
        if (!LEVEL1) {
            const float2 *pl = reinterpret_cast<const float2 *>(row.l + q2);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 u = __ldg(pl + j);
                w[2 * j] = u.x;
                w[2 * j + 1] = u.y;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            v[k] = __ldg(row.h + L.col[k]);
            if (!LEVEL1) w[k] = __ldg(row.l + L.col[k]);
        }
    }
}

template <bool LEVEL1>
__device__ __forceinline__ void row_item(const AnaArgs &a, const RowIn &row, const Lane<LEVEL1> &L, int q2,
                                         float &rh, float &rl, float &s, float &t) {
    float v[8], w[8];
    row_load<LEVEL1>(row, L, q2, v, w);
    row_math<LEVEL1>(a.f, v, w, rh, rl, s, t);
}

// Level-1 input ring: interior warps stage their 72 input columns of each
// input row in a per-warp ring of 24 rows with cp.async, 4-row chunks issued
// 16 rows ahead of use, so the global latency overlaps the filter arithmetic.
constexpr int kRingRows = 24, kRingCols = 72, kChunk = 4;
__device__ __forceinline__ void ring_cp16(float *dst, const float *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void ring_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void ring_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <bool LEVEL1, class T, int SP, int WARPS>
__global__ void __launch_bounds__(32 * WARPS, 24 / WARPS) k_analysis_stream(AnaArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int plane = blockIdx.z;
    const int R2 = a.R >> 1, C2 = a.Cc >> 1;
    const int cq0 = (blockIdx.x * WARPS + warp) * 32;  // first output column of this warp
    if (cq0 >= C2) return;                             // whole warp past the plane
    const int p0 = blockIdx.y * SP;
    const int q = min(cq0 + lane, C2 - 1);             // lanes past the edge recompute the last column
    const bool store_q = cq0 + lane < C2;
    const int srcH = LEVEL1 ? a.H : a.R, srcW = LEVEL1 ? a.W : a.Cc;
    const long long pbase = (long long)plane * srcH * srcW;

    Lane<LEVEL1> L;
    {
        const int qmax = min(cq0 + 31, C2 - 1);
        const bool aligned8 = ((reinterpret_cast<uintptr_t>(a.inh) |
                                (LEVEL1 ? (uintptr_t)0 : reinterpret_cast<uintptr_t>(a.inl))) & 7u) == 0;
        L.fast = (2 * qmax + 7 < srcW) && ((srcW & 1) == 0) && aligned8;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int gx = wrap_near(2 * q + k, a.Cc);
            L.col[k] = LEVEL1 ? mirror(gx, a.W) : gx;
            if (!PRNU_DCHECK(L.col[k] >= 0 && L.col[k] < srcW, L.col[k])) L.col[k] = 0;
        }
    }
    auto row_at = [&](int y) {
        const int gy = wrap_near(y, a.R);
        int sy = LEVEL1 ? mirror(gy, a.H) : gy;
        if (!PRNU_DCHECK(sy >= 0 && sy < srcH, sy)) sy = 0;
        RowIn r;
        r.h = a.inh + pbase + (long long)sy * srcW;
        r.l = LEVEL1 ? nullptr : a.inl + pbase + (long long)sy * srcW;
        return r;
    };
    const float scale = a.scale_on ? __frcp_rn((float)a.sc.count(plane)) : 1.f;

    // ring: level 1, interior warps whose 72-column window stays inside the row
    constexpr bool RING_OK = LEVEL1 && WARPS <= 4;
    __shared__ __align__(16) float ring[RING_OK ? WARPS : 1][RING_OK ? kRingRows : 1][RING_OK ? kRingCols : 4];
    const bool use_ring = RING_OK && L.fast && 2 * cq0 + kRingCols <= srcW && (srcW & 3) == 0 &&
                          ((reinterpret_cast<uintptr_t>(a.inh) & 15u) == 0);
    float *const rbase = &ring[RING_OK ? warp : 0][0][0];
    const int y0 = 2 * p0;
    const int pend = min(p0 + SP, R2);
    const int t_last = 2 * (pend - p0) + 5;  // last strip-relative input row used
    // chunk c holds strip rows 4c .. 4c+3 (skipped past t_last; an empty group keeps the count)
    auto issue_chunk = [&](int c) {
        if (RING_OK && use_ring && kChunk * c <= t_last) {
            for (int it = lane; it < kChunk * (kRingCols / 4); it += 32) {
                const int r = kChunk * c + it / (kRingCols / 4), j = it % (kRingCols / 4);
                if (!PRNU_DCHECK(2 * cq0 + 4 * j + 3 < srcW, 2 * cq0 + 4 * j)) continue;
                ring_cp16(rbase + (r % kRingRows) * kRingCols + 4 * j, row_at(y0 + r).h + 2 * cq0 + 4 * j);
            }
        }
        ring_commit();
    };
    auto ring_row = [&](int t, float &rh_, float &rl_, float &rs_, float &rt_) {
        const float2 *pr = reinterpret_cast<const float2 *>(rbase + (t % kRingRows) * kRingCols + 2 * lane);
        float v[8], w[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 u = pr[k];
            v[2 * k] = u.x;
            v[2 * k + 1] = u.y;
        }
        row_math<LEVEL1>(a.f, v, w, rh_, rl_, rs_, rt_);
    };

    float rh[8], rl[8], rs[8], rt[8];
    if (use_ring) {
        for (int c = 0; c < 4; ++c) issue_chunk(c);  // strip rows 0..15
        ring_wait<2>();                                 // rows 0..7 have landed
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 6; ++k) ring_row(k, rh[k], rl[k], rs[k], rt[k]);
    } else {
#pragma unroll
        for (int k = 0; k < 6; ++k) row_item<LEVEL1>(a, row_at(y0 + k), L, 2 * q, rh[k], rl[k], rs[k], rt[k]);
    }

    for (int pb = p0, m = 0; pb < pend; pb += 4, ++m) {
        if (use_ring) {
            // iteration m reads strip rows 8m+6 .. 8m+13 (chunks <= 2m+3); chunks
            // 2m+4, 2m+5 (rows 8m+16 .. 8m+23) reuse the slots of rows 8m-8 ..
            // 8m-1, all read before this point
            __syncwarp();
            issue_chunk(2 * m + 4);
            issue_chunk(2 * m + 5);
            ring_wait<2>();
            __syncwarp();
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int p = pb + j;
            // input rows 2p+6, 2p+7 go to slots (2j+6) mod 8, (2j+7) mod 8
            const int s6 = (2 * j + 6) & 7, s7 = (2 * j + 7) & 7;
            if (use_ring) {
                ring_row(2 * (p - p0) + 6, rh[s6], rl[s6], rs[s6], rt[s6]);
                ring_row(2 * (p - p0) + 7, rh[s7], rl[s7], rs[s7], rt[s7]);
            } else {
                row_item<LEVEL1>(a, row_at(2 * p + 6), L, 2 * q, rh[s6], rl[s6], rs[s6], rt[s6]);
                row_item<LEVEL1>(a, row_at(2 * p + 7), L, 2 * q, rh[s7], rl[s7], rs[s7], rt[s7]);
            }
            // column pass over rows 2p..2p+7 = slots 2j .. 2j+7 (mod 8)
            if (p < pend && store_q && PRNU_DCHECK(p < R2 && q < C2 && plane < a.P, (long long)p * C2 + q))
                col_store<LEVEL1, T>(a, rh, rl, rs, rt, (2 * j) & 7, ((long long)plane * R2 + p) * C2 + q, scale);
        }
    }
    if (use_ring) ring_wait<0>();  // no copy outstanding at exit
}

constexpr int TP = 16, TQ = 32;                 // output tile: TP rows x TQ cols
constexpr int IR = 2 * TP + 6, IC = 2 * TQ + 6;  // input tile with the 6-sample halo
constexpr int ICS = IC + 2;                      // even row stride: float2-aligned rows
constexpr int NCOL = (IC + 31) / 32;             // input columns per thread

template <bool LEVEL1, class T>
__global__ void __launch_bounds__(256, 5) k_analysis(AnaArgs a) {
    __shared__ __align__(16) float vh[IR][ICS];
    __shared__ __align__(16) float vl[LEVEL1 ? 1 : IR][LEVEL1 ? 2 : ICS];
    __shared__ float rh[IR][TQ + 1], rl[LEVEL1 ? 1 : IR][LEVEL1 ? 1 : TQ + 1];
    __shared__ float ss[IR][TQ + 1], tt[IR][TQ + 1];

    const int plane = blockIdx.z;
    const int p0 = blockIdx.y * TP, q0 = blockIdx.x * TQ;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int R2 = a.R >> 1, C2 = a.Cc >> 1;

    // 1) input tile: periodic wrap in the (padded) domain; level 1 mirrors the
    //    padded index into the unpadded source.  Column sources are computed
    //    once per thread, row sources once per row.
    int srcx[NCOL];
#pragma unroll
    for (int k = 0; k < NCOL; ++k) {
        const int c = tx + 32 * k;
        const int gx = wrap_near(2 * q0 + c, a.Cc);
        srcx[k] = LEVEL1 ? mirror(gx, a.W) : gx;
    }
    const int srcH = LEVEL1 ? a.H : a.R, srcW = LEVEL1 ? a.W : a.Cc;
    // above level 1, tiles whose ICS columns lie inside the row (no wrap)
    // arrive as 16-byte copies of both parts
    const bool chunks = !LEVEL1 && (srcW & 3) == 0 && 2 * q0 + ICS <= srcW &&
                        ((reinterpret_cast<uintptr_t>(a.inh) | reinterpret_cast<uintptr_t>(a.inl)) & 15u) == 0;
    if (chunks) {
        const int tid = ty * 32 + tx;
        for (int it = tid; it < IR * (ICS / 4); it += 256) {
            const int r = it / (ICS / 4), j = it - r * (ICS / 4);
            const int sy = wrap_near(2 * p0 + r, a.R);
            const long long off = ((long long)plane * srcH + sy) * srcW + 2 * q0 + 4 * j;
            if (!PRNU_DCHECK(sy >= 0 && sy < srcH && 2 * q0 + 4 * j + 3 < srcW, off)) continue;
            ring_cp16(&vh[r][4 * j], a.inh + off);
            if (!LEVEL1) ring_cp16(&vl[r][4 * j], a.inl + off);
        }
        ring_commit();
        ring_wait<0>();
    } else {
        for (int r = ty; r < IR; r += 8) {
            const int gy = wrap_near(2 * p0 + r, a.R);
            const int sy = LEVEL1 ? mirror(gy, a.H) : gy;
            const long long rowoff = ((long long)plane * srcH + sy) * srcW;
#pragma unroll
            for (int k = 0; k < NCOL; ++k) {
                const int c = tx + 32 * k;
                if (c < IC && PRNU_DCHECK(sy >= 0 && sy < srcH && srcx[k] >= 0 && srcx[k] < srcW, rowoff + srcx[k])) {
                    vh[r][c] = __ldg(a.inh + rowoff + srcx[k]);
                    if (!LEVEL1) vl[r][c] = __ldg(a.inl + rowoff + srcx[k]);
                }
            }
        }
    }
    __syncthreads();

    // 2) row pass on differences; thread tx owns output column q = tx and reads
    //    the 8 input samples 2q..2q+7 as four float2 (conflict-free)
    {
        const int q = tx;
        for (int r = ty; r < IR; r += 8) {
            float v[8], w[8];
            const float2 *row = reinterpret_cast<const float2 *>(&vh[r][0]);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 t = row[q + j];
                v[2 * j] = t.x;
                v[2 * j + 1] = t.y;
            }
            if (!LEVEL1) {
                const float2 *rowl = reinterpret_cast<const float2 *>(&vl[r][0]);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float2 t = rowl[q + j];
                    w[2 * j] = t.x;
                    w[2 * j + 1] = t.y;
                }
            }
            float h0, l0, s, t;
            row_math<LEVEL1>(a.f, v, w, h0, l0, s, t);
            rh[r][q] = h0;
            if (!LEVEL1) rl[r][q] = l0;
            ss[r][q] = s;
            tt[r][q] = t;
        }
    }
    __syncthreads();

    // 3) column pass: thread (tx, ty) owns output rows 2ty, 2ty+1 of column q =
    //    tx, which read input rows 4ty .. 4ty+9 (six of them shared), each read
    //    once from shared memory
    const float scale = a.scale_on ? __frcp_rn((float)a.sc.count(plane)) : 1.f;
    const int q = tx, qq = q0 + q;
    float ch[10], cl[10], cs[10], ct[10];
#pragma unroll
    for (int j = 0; j < 10; ++j) {
        const int y = 4 * ty + j;
        ch[j] = rh[y][q];
        cl[j] = LEVEL1 ? 0.f : rl[y][q];
        cs[j] = ss[y][q];
        ct[j] = tt[y][q];
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int p = p0 + 2 * ty + e;
        if (p >= R2 || qq >= C2) continue;
        const float r0h = ch[2 * e];
        const float r0l = cl[2 * e];
        pf2 AB = pf2_of(0.f, 0.f), S = pf2_of(0.f, 0.f), Tp = pf2_of(0.f, 0.f);  // {A, B}, {Sh, Sg}, {Th, Tg}
#pragma unroll
        for (int j = 1; j < kTaps; ++j) {
            float D = __fsub_rn(ch[2 * e + j], r0h);
            if (!LEVEL1) D = __fadd_rn(D, __fsub_rn(cl[2 * e + j], r0l));
            AB = pf2_fma(hg_of(a.f, j), pf2_of(D, D), AB);
        }
#pragma unroll
        for (int j = 0; j < kTaps; ++j) {
            const float sv = cs[2 * e + j], tv = ct[2 * e + j];
            S = pf2_fma(hg_of(a.f, j), pf2_of(sv, sv), S);
            Tp = pf2_fma(hg_of(a.f, j), pf2_of(tv, tv), Tp);
        }
        float A, B, Sh, Sg, Th, Tg;
        pf2_split(AB, A, B);
        pf2_split(S, Sh, Sg);
        pf2_split(Tp, Th, Tg);
        const float llsmall = __fmaf_rn(kSqrt2f, A, Sh);
        const float lh = __fmaf_rn(kSqrt2f, B, Sg);
        const long long o = ((long long)plane * R2 + p) * C2 + qq;
        if (a.LLh) {
            float sh, se, lo;
            two_sum(2.f * r0h, llsmall, sh, se);
            lo = __fadd_rn(2.f * r0l, se);
            float hh, ll;
            fast_two_sum(sh, lo, hh, ll);
            a.LLh[o] = hh;
            a.LLl[o] = ll;
        }
        stf<T>(static_cast<T *>(a.LH) + o, lh * scale);
        stf<T>(static_cast<T *>(a.HL) + o, Th * scale);
        stf<T>(static_cast<T *>(a.HH) + o, Tg * scale);
    }
}

template <class T, int SP, int WARPS, bool LEVEL1 = true>
static void launch_stream(const AnaArgs &a, cudaStream_t st) {
    dim3 block(32 * WARPS);
    dim3 grid((unsigned)((a.Cc / 2 + 32 * WARPS - 1) / (32 * WARPS)), (unsigned)((a.R / 2 + SP - 1) / SP),
              (unsigned)a.P);
    k_analysis_stream<LEVEL1, T, SP, WARPS><<<grid, block, 0, st>>>(a);
}

template <class T>
static void launch_analysis_t(const AnaArgs &a, bool level1, int shape, cudaStream_t st) {
    if (level1) {
        switch (shape) {
            case 0: launch_stream<T, 16, 4>(a, st); break;
            case 2: launch_stream<T, 64, 4>(a, st); break;
            case 3: launch_stream<T, 32, 2>(a, st); break;
            case 4: launch_stream<T, 32, 8>(a, st); break;
            case 5: launch_stream<T, 64, 2>(a, st); break;
            default: launch_stream<T, 32, 4>(a, st); break;
        }
    } else if (shape == 1) {
        launch_stream<T, 16, 4, false>(a, st);
    } else if (shape == 2) {
        launch_stream<T, 32, 2, false>(a, st);
    } else {
        dim3 block(32, 8);
        dim3 grid((unsigned)((a.Cc / 2 + TQ - 1) / TQ), (unsigned)((a.R / 2 + TP - 1) / TP), (unsigned)a.P);
        k_analysis<false, T><<<grid, block, 0, st>>>(a);
    }
}

cudaError_t launch_analysis(const AnaArgs &a, bool level1, cudaStream_t st, int shape) {
    if (a.sdt == SB_F16)
        launch_analysis_t<__half>(a, level1, shape, st);
    else if (a.sdt == SB_BF16)
        launch_analysis_t<__nv_bfloat16>(a, level1, shape, st);
    else
        launch_analysis_t<float>(a, level1, shape, st);
    return cudaGetLastError();
}

}  // namespace prnu
