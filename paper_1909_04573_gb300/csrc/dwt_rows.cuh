// dwt_rows.cuh -- the per-sample arithmetic of one analysis level in
// difference form (the derivation is at the top of k_dwt.cu): the row pass of
// one input row and the column pass plus subband stores of one output
// coefficient.  Shared by the streaming analysis (k_dwt.cu) and the fused
// group-sum + level-1 kernel (k_sda_dwt.cu), so both produce the same bits.
#pragma once

#include "kernels.cuh"

namespace prnu {

constexpr float kSqrt2f = 1.41421356237309504880f;

// row pass of one input row from its samples 2q..2q+7 (v: high parts, w: low
// parts above level 1): ref, s = sum_{k>=1} h_k (v_k - v_0), t = sum g_k (v_k - v_0)
template <bool LEVEL1>
__device__ __forceinline__ void row_math(const Filt &f, const float *v, const float *w, float &rh, float &rl,
                                         float &s, float &t) {
    pf2 st = pf2_of(0.f, 0.f);  // {s, t}
#pragma unroll
    for (int k = 1; k < kTaps; ++k) {
        float dlt = __fsub_rn(v[k], v[0]);
        if (!LEVEL1) dlt = __fadd_rn(dlt, __fsub_rn(w[k], w[0]));
        st = pf2_fma(hg_of(f, k), pf2_of(dlt, dlt), st);
    }
    rh = v[0];
    rl = LEVEL1 ? 0.f : w[0];
    pf2_split(st, s, t);
}

// Column pass over the row-pass results of input rows 2p..2p+7, held in an
// 8-slot ring starting at slot b0 (a compile-time constant after unrolling),
// and the stores of output o: LL as a float-float pair in sum units (when
// a.LLh is set), LH / HL / HH scaled by `scale`.
template <bool LEVEL1, class T>
__device__ __forceinline__ void col_store(const AnaArgs &a, const float *rh, const float *rl, const float *rs,
                                          const float *rt, int b0, long long o, float scale) {
    const float r0h = rh[b0], r0l = rl[b0];
    pf2 AB = pf2_of(0.f, 0.f), S = pf2_of(0.f, 0.f), Tp = pf2_of(0.f, 0.f);  // {A, B}, {Sh, Sg}, {Th, Tg}
#pragma unroll
    for (int k = 1; k < kTaps; ++k) {
        const int sl = (b0 + k) & 7;
        float D = __fsub_rn(rh[sl], r0h);
        if (!LEVEL1) D = __fadd_rn(D, __fsub_rn(rl[sl], r0l));
        AB = pf2_fma(hg_of(a.f, k), pf2_of(D, D), AB);
    }
#pragma unroll
    for (int k = 0; k < kTaps; ++k) {
        const int sl = (b0 + k) & 7;
        S = pf2_fma(hg_of(a.f, k), pf2_of(rs[sl], rs[sl]), S);
        Tp = pf2_fma(hg_of(a.f, k), pf2_of(rt[sl], rt[sl]), Tp);
    }
    float A, B, Sh, Sg, Th, Tg;
    pf2_split(AB, A, B);
    pf2_split(S, Sh, Sg);
    pf2_split(Tp, Th, Tg);
    const float llsmall = __fmaf_rn(kSqrt2f, A, Sh);
    const float lh = __fmaf_rn(kSqrt2f, B, Sg);
    if (a.LLh) {
        float sh, se;
        two_sum(2.f * r0h, llsmall, sh, se);
        const float lo = __fadd_rn(2.f * r0l, se);
        float hh, ll;
        fast_two_sum(sh, lo, hh, ll);
        a.LLh[o] = hh;
        a.LLl[o] = ll;
    }
    stf<T>(static_cast<T *>(a.LH) + o, lh * scale);
    stf<T>(static_cast<T *>(a.HL) + o, Th * scale);
    stf<T>(static_cast<T *>(a.HH) + o, Tg * scale);
}

}  // namespace prnu
