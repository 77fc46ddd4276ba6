// k_sda.cu -- SDA frames (Sec. III-B): exact per-group sums of uint8 frames.
//
// A frame row is W*C interleaved bytes.  A block owns a segment of SEGPX
// pixels of one row of one group (SEGPX*C bytes, a multiple of 16) and each
// thread one 16-byte chunk of it, read from every frame of the group with one
// 16-byte streaming (evict-first) load per frame, so each warp load is 512
// contiguous bytes.  The bytes are summed exactly: two 16-bit lanes per
// 32-bit register hold the even and odd bytes of each loaded word (a lane
// holds at most 256 * 255 < 2^16) and are flushed into 32-bit totals every 256
// frames.  The totals go through shared memory, where the interleaved byte
// order is transposed, so each channel plane is written with consecutive
// threads on consecutive pixels.  Output: float32 (exact below 2^24, i.e.
// groups of up to 65793 frames), planar [group][C][H][W], as sums (the
// fingerprint pipeline stays in "sum units" until the details are formed) or
// as correctly rounded means.  Frames may also be float16 (one 16-byte load
// per frame then carries 8 values, summed in float32; such sums are not exact
// integers, but the same pipeline applies).
#include <algorithm>

#include "kernels.cuh"

namespace prnu {

__device__ __forceinline__ void acc_word(uint32_t v, uint32_t &ev, uint32_t &od) {
    ev += v & 0x00FF00FFu;
    od += (v >> 8) & 0x00FF00FFu;
}

// Frames ahead whose row segment thread 0 of a block requests into L2 with a
// bulk prefetch (fire and forget: no completion, no wait), so that the
// block's 16-byte loads find their data in L2.  Sizes are rounded down to 16
// bytes, so a prefetch never reaches past the segment.
constexpr int kPrefetch = 8;
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <int C, int SEGPX, bool MULTI>
__global__ void __launch_bounds__(SEGPX * C / 16) k_sda_sum(SdaArgs a) {
    constexpr int NT = SEGPX * C / 16;  // threads = 16-byte chunks per segment
    __shared__ float sbuf[SEGPX * C];
    const int rowbytes = a.W * C;
    const int nseg = (a.W + SEGPX - 1) / SEGPX;
    const long long units = (long long)a.G * a.H * nseg;
    const long long plane = (long long)a.H * a.W;
    const int k = threadIdx.x;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        const int seg = (int)(u % nseg);
        const long long r = u / nseg;
        const int y = (int)(r % a.H);
        const int gi = (int)(r / a.H);
        int j0, j1;
        const uint8_t *fr = a.frames;
        long long fstride = a.frame_stride, rpitch = a.row_pitch;
        if (MULTI) {  // multi-camera pass: the group's own frames
            const GroupDesc &gdesc = a.gd[gi];
            fr = gdesc.frames;
            fstride = gdesc.frame_stride;
            rpitch = gdesc.row_pitch;
            j0 = 0;
            j1 = gdesc.n;
        } else {
            const int g = a.g0 + gi;
            j0 = g * a.d;
            j1 = min(a.m, j0 + a.d);
        }
        const bool al16 = ((reinterpret_cast<uintptr_t>(fr) | (uintptr_t)fstride | (uintptr_t)rpitch) & 15u) == 0;
        const int x0 = seg * SEGPX;
        const int npx = min(SEGPX, a.W - x0);
        const int b0 = x0 * C + 16 * k;
        const int nb = PRNU_DCHECK(y < a.H && gi < a.G && j1 <= (MULTI ? a.gd[gi].n : a.m), u) ? min(16, rowbytes - b0)
                                                                                            : 0;
        uint32_t tot[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) tot[i] = 0;
        if (nb > 0) {
            const uint8_t *base = fr + (long long)y * rpitch + b0;
            if (al16 && nb == 16) {
                // thread 0 asks L2 for the segment kPrefetch frames ahead
                const uint8_t *seg = fr + (long long)y * rpitch + (long long)x0 * C;
                const unsigned segb = (unsigned)(min(SEGPX * C, rowbytes - x0 * C) & ~15);
                for (int jb = j0; jb < j1; jb += 256) {
                    const int je = min(j1, jb + 256);
                    uint32_t ev[4] = {0, 0, 0, 0}, od[4] = {0, 0, 0, 0};
                    const uint8_t *p = base + (long long)jb * fstride;
#pragma unroll 4
                    for (int j = jb; j < je; ++j, p += fstride) {
                        if (k == 0 && j + kPrefetch < j1 && segb) prefetch_l2(seg + (long long)(j + kPrefetch) * fstride, segb);
                        const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(p));
                        acc_word(v.x, ev[0], od[0]);
                        acc_word(v.y, ev[1], od[1]);
                        acc_word(v.z, ev[2], od[2]);
                        acc_word(v.w, ev[3], od[3]);
                    }
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        tot[4 * w + 0] += ev[w] & 0xFFFFu;
                        tot[4 * w + 1] += od[w] & 0xFFFFu;
                        tot[4 * w + 2] += ev[w] >> 16;
                        tot[4 * w + 3] += od[w] >> 16;
                    }
                }
            } else {
                for (int j = j0; j < j1; ++j) {
                    const uint8_t *p = base + (long long)j * fstride;
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (i < nb) tot[i] += p[i];
                }
            }
        }
        const float fn = (float)(j1 - j0);
        if (u != blockIdx.x) __syncthreads();  // the previous unit's readers are done
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float s = (float)tot[i];
            sbuf[16 * k + i] = a.mean ? __fdiv_rn(s, fn) : s;
        }
        __syncthreads();
        float *o = a.out + (long long)gi * C * plane + (long long)y * a.W + x0;
#pragma unroll
        for (int c = 0; c < C; ++c)
            for (int x = k; x < npx; x += NT)
                if (PRNU_DCHECK(x0 + x < a.W, x0 + x)) o[(long long)c * plane + x] = sbuf[x * C + c];
    }
}

// float16 frames: a thread owns 8 consecutive values (16 bytes) of a row
// segment and sums them in float32 over the group's frames.
template <int C, int SEGPX, bool MULTI>
__global__ void __launch_bounds__(SEGPX * C / 8) k_sda_sum_f16(SdaArgs a) {
    constexpr int NT = SEGPX * C / 8;
    __shared__ float sbuf[SEGPX * C];
    const int rowvals = a.W * C;
    const int nseg = (a.W + SEGPX - 1) / SEGPX;
    const long long units = (long long)a.G * a.H * nseg;
    const long long plane = (long long)a.H * a.W;
    const int k = threadIdx.x;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        const int seg = (int)(u % nseg);
        const long long r = u / nseg;
        const int y = (int)(r % a.H);
        const int gi = (int)(r / a.H);
        int j0, j1;
        const uint8_t *fr = a.frames;
        long long fstride = a.frame_stride, rpitch = a.row_pitch;
        if (MULTI) {
            const GroupDesc &gdesc = a.gd[gi];
            fr = gdesc.frames;
            fstride = gdesc.frame_stride;
            rpitch = gdesc.row_pitch;
            j0 = 0;
            j1 = gdesc.n;
        } else {
            const int g = a.g0 + gi;
            j0 = g * a.d;
            j1 = min(a.m, j0 + a.d);
        }
        const bool al16 = ((reinterpret_cast<uintptr_t>(fr) | (uintptr_t)fstride | (uintptr_t)rpitch) & 15u) == 0;
        const int x0 = seg * SEGPX;
        const int npx = min(SEGPX, a.W - x0);
        const int e0 = x0 * C + 8 * k;  // first value of this thread's chunk
        const int ne = min(8, rowvals - e0);
        float tot[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) tot[i] = 0.f;
        if (ne > 0) {
            const uint8_t *base = fr + (long long)y * rpitch + 2LL * e0;
            if (al16 && ne == 8) {
                const uint8_t *seg = fr + (long long)y * rpitch + 2LL * x0 * C;
                const unsigned segb = (unsigned)(min(SEGPX * C, rowvals - x0 * C) * 2 & ~15);
#pragma unroll 4
                for (int j = j0; j < j1; ++j) {
                    if (k == 0 && j + kPrefetch < j1 && segb) prefetch_l2(seg + (long long)(j + kPrefetch) * fstride, segb);
                    const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(base + (long long)j * fstride));
                    const __half2 *h2 = reinterpret_cast<const __half2 *>(&v);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float2 f = __half22float2(h2[i]);
                        tot[2 * i] += f.x;
                        tot[2 * i + 1] += f.y;
                    }
                }
            } else {
                for (int j = j0; j < j1; ++j) {
                    const __half *p = reinterpret_cast<const __half *>(base + (long long)j * fstride);
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (i < ne) tot[i] += __half2float(p[i]);
                }
            }
        }
        const float fn = (float)(j1 - j0);
        if (u != blockIdx.x) __syncthreads();
#pragma unroll
        for (int i = 0; i < 8; ++i) sbuf[8 * k + i] = a.mean ? __fdiv_rn(tot[i], fn) : tot[i];
        __syncthreads();
        float *o = a.out + (long long)gi * C * plane + (long long)y * a.W + x0;
#pragma unroll
        for (int c = 0; c < C; ++c)
            for (int x = k; x < npx; x += NT) o[(long long)c * plane + x] = sbuf[x * C + c];
    }
}

__global__ void k_put_desc(PassDesc pd, PassDesc *dst) {
    // one block copies the by-value descriptor into device memory
    const int *src = reinterpret_cast<const int *>(&pd);
    int *out = reinterpret_cast<int *>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(PassDesc) / sizeof(int)); i += blockDim.x) out[i] = src[i];
}

cudaError_t launch_put_desc(const PassDesc &pd, PassDesc *dst, cudaStream_t st) {
    k_put_desc<<<1, 256, 0, st>>>(pd, dst);
    return cudaGetLastError();
}


cudaError_t launch_sda(const SdaArgs &a, int num_sms, cudaStream_t st) {
    if (a.frame_half) {
        constexpr int SEG = 1024;
        const long long units = (long long)a.G * a.H * ((a.W + SEG - 1) / SEG);
        if (a.C == 3) {
            constexpr int NT = SEG * 3 / 8;
            const long long blocks = std::min<long long>(units, (long long)num_sms * (a.blocks_per_sm > 0 ? a.blocks_per_sm : 2048 / NT));
            if (a.gd)
                k_sda_sum_f16<3, SEG, true><<<(unsigned)std::max<long long>(blocks, 1), NT, 0, st>>>(a);
            else
                k_sda_sum_f16<3, SEG, false><<<(unsigned)std::max<long long>(blocks, 1), NT, 0, st>>>(a);
        } else {
            constexpr int NT = SEG / 8;
            const long long blocks = std::min<long long>(units, (long long)num_sms * (a.blocks_per_sm > 0 ? a.blocks_per_sm : 2048 / NT));
            if (a.gd)
                k_sda_sum_f16<1, SEG, true><<<(unsigned)std::max<long long>(blocks, 1), NT, 0, st>>>(a);
            else
                k_sda_sum_f16<1, SEG, false><<<(unsigned)std::max<long long>(blocks, 1), NT, 0, st>>>(a);
        }
        return cudaGetLastError();
    }
    if (a.C == 3) {
        constexpr int SEG = 1024, NT = SEG * 3 / 16;
        const long long units = (long long)a.G * a.H * ((a.W + SEG - 1) / SEG);
        const long long blocks = std::min<long long>(units, (long long)num_sms * (a.blocks_per_sm > 0 ? a.blocks_per_sm : 2048 / NT));
        if (a.gd)
            k_sda_sum<3, SEG, true><<<(unsigned)std::max<long long>(blocks, 1), NT, 0, st>>>(a);
        else
            k_sda_sum<3, SEG, false><<<(unsigned)std::max<long long>(blocks, 1), NT, 0, st>>>(a);
    } else {
        constexpr int SEG = 4096, NT = SEG / 16;
        const long long units = (long long)a.G * a.H * ((a.W + SEG - 1) / SEG);
        const long long blocks = std::min<long long>(units, (long long)num_sms * (a.blocks_per_sm > 0 ? a.blocks_per_sm : 2048 / NT));
        if (a.gd)
            k_sda_sum<1, SEG, true><<<(unsigned)std::max<long long>(blocks, 1), NT, 0, st>>>(a);
        else
            k_sda_sum<1, SEG, false><<<(unsigned)std::max<long long>(blocks, 1), NT, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace prnu
