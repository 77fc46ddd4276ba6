// common.cuh -- shared device/host helpers of libprnu (GB300, sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/prnu.h"
#include "debug.cuh"

namespace prnu {

constexpr int kTaps = 8;       // 8-tap Daubechies (4 vanishing moments)
constexpr int kMaxLevels = 6;
constexpr int kMaxRadius = 4;  // windows up to 9 x 9

// Filter bank in float32, passed by value to kernels (kernel parameters live
// in the constant bank).  g[k] = (-1)^k h[7-k].
struct Filt {
    __align__(8) float h[kTaps];
    __align__(8) float g[kTaps];
    __align__(8) float hg[kTaps][2];  // (h[k], g[k]) side by side, for packed float32x2 arithmetic
};

// ---- packed float32x2 FMA (Blackwell): two independent round-to-nearest
// FMAs in one instruction, so the bits equal those of two scalar __fmaf_rn.
using pf2 = unsigned long long;  // {lo lane, hi lane}
__device__ __forceinline__ pf2 pf2_of(float a, float b) {
    pf2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void pf2_split(pf2 v, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ pf2 pf2_fma(pf2 a, pf2 b, pf2 c) {
    pf2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ pf2 pf2_at(const float *p) { return *reinterpret_cast<const pf2 *>(p); }  // 8-byte aligned
// analysis: the low- and high-pass accumulators of one output advance together,
// {x, y} += {h_k, g_k} * {d, d}
__device__ __forceinline__ pf2 hg_of(const Filt &f, int k) { return pf2_at(&f.hg[k][0]); }
// synthesis of an output pair: v_e = sum_{t=0..3} h[e+2t] x[t] + g[e+2t] y[t]
// (in that order) for e = 0, 1, as {v_0, v_1} += {h[2t], h[2t+1]} * {x[t], x[t]}, ...
__device__ __forceinline__ void synth_pair2(const Filt &f, const float *x, const float *y, float &v0, float &v1) {
    pf2 acc = pf2_of(0.f, 0.f);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        acc = pf2_fma(pf2_at(&f.h[2 * t]), pf2_of(x[t], x[t]), acc);
        acc = pf2_fma(pf2_at(&f.g[2 * t]), pf2_of(y[t], y[t]), acc);
    }
    pf2_split(acc, v0, v1);
}

// Local-variance windows.
struct Win {
    int n;
    int r[4];       // radii (w-1)/2
    float inv[4];   // 1/w^2
};

// One SDA group of a multi-camera pass: its first frame, strides, frame
// count and camera index.
struct GroupDesc {
    const uint8_t *frames;
    long long frame_stride, row_pitch;
    int n, cam;
};
struct CamDesc {
    float *num, *den;
};
constexpr int kMaxPassGroups = 192;
constexpr int kMaxPassCams = 64;
// Passed to one small kernel by value (graph-capturable), which writes it to
// the workspace for the kernels of the pass.
struct PassDesc {
    int G, ncam;
    GroupDesc g[kMaxPassGroups];
    CamDesc cam[kMaxPassCams];
};

// Per-plane count of frames averaged into the plane: plane p belongs to image
// g0 + p / C, whose frame count is min(d, m - image*d), or, in a
// multi-camera pass, the count recorded for that group.  Details are scaled
// by 1/count (group sums are kept exact, in "sum units", through the LL chain).
struct PlaneScale {
    int d, m, g0, C;
    const GroupDesc *gd;  // null: single sequence
    __device__ __forceinline__ int count(int plane) const {
        if (gd) return gd[plane / C].n;
        int img = g0 + plane / C;
        int left = m - img * d;
        return left < d ? left : d;
    }
};

__host__ __device__ __forceinline__ int wrap(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

// Periodic index for i within one period of [0, n) (the common case of a
// tile's halo): two compare-and-adds; falls back to a modulo otherwise
// (planes smaller than a tile's reach).
__host__ __device__ __forceinline__ int wrap_near(int i, int n) {
    if (i < 0) i += n;
    if (i >= n) i -= n;
    if (i < 0 || i >= n) i = wrap(i, n);
    return i;
}

// Mirror padding with edge repeat: index in [0, 2n) -> [0, n).
__host__ __device__ __forceinline__ int mirror(int i, int n) { return i < n ? i : 2 * n - 1 - i; }

// ---- error-free float transformations (float-float pairs) -----------------
// TwoSum (Knuth): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// FastTwoSum (Dekker), requires |a| >= |b| or a == 0.
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void ff_add(float &hi, float &lo, float v) {
    float s, e;
    two_sum(hi, v, s, e);
    hi = s;
    lo = __fadd_rn(lo, e);
}

// ---- storage types of the detail / noise subbands (arithmetic is float32) --
enum SubbandType : int { SB_F32 = 0, SB_F16 = 1, SB_BF16 = 2 };

__host__ __device__ inline size_t subband_bytes(int sdt) { return sdt == SB_F32 ? 4 : 2; }

template <class T> __device__ __forceinline__ float ldf(const T *p);
template <> __device__ __forceinline__ float ldf<float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ float ldf<__half>(const __half *p) { return __half2float(__ldg(p)); }
template <> __device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16 *p) {
    return __bfloat162float(__ldg(p));
}
template <class T> __device__ __forceinline__ void stf(T *p, float v);
template <> __device__ __forceinline__ void stf<float>(float *p, float v) { *p = v; }
template <> __device__ __forceinline__ void stf<__half>(__half *p, float v) { *p = __float2half_rn(v); }
template <> __device__ __forceinline__ void stf<__nv_bfloat16>(__nv_bfloat16 *p, float v) {
    *p = __float2bfloat16_rn(v);
}

// float-float accumulation (compensated, Neumaier form via TwoSum):
// (hi, lo) += v with the rounding error of the add kept in lo.
__device__ __forceinline__ void ff_add(float &hi, float &lo, float v);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace prnu
