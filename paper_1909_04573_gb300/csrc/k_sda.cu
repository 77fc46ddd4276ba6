// k_sda.cu -- SDA frames (Sec. IV-B): exact per-group sums of uint8 frames.
//
// A frame row is W*C interleaved bytes.  One thread owns a 16-byte chunk of
// one row of one group and reads that chunk from every frame of the group
// with one 16-byte streaming (evict-first) load per frame, so each warp load
// is 512 contiguous bytes.  The bytes are summed exactly: two 16-bit lanes per
// 32-bit register hold the even and odd bytes of each loaded word (a lane
// holds at most 256 * 255 < 2^16) and are flushed into 32-bit totals every 256
// frames.  Only at write-out is a byte position mapped to (pixel, channel).
// The sums go out as float32 (exact below 2^24, i.e. groups of up to 65793
// frames) in planar [group][C][H][W] layout: as sums (the fingerprint
// pipeline stays in "sum units" until the details are formed) or as
// correctly rounded means.
#include "kernels.cuh"

namespace prnu {

__device__ __forceinline__ void acc_word(uint32_t v, uint32_t &ev, uint32_t &od) {
    ev += v & 0x00FF00FFu;
    od += (v >> 8) & 0x00FF00FFu;
}

__global__ void __launch_bounds__(256) k_sda_sum(SdaArgs a) {
    const int rowbytes = a.W * a.C;
    const int chunks = (rowbytes + 15) >> 4;
    const long long units = (long long)a.G * a.H * chunks;
    const bool aligned16 = ((reinterpret_cast<uintptr_t>(a.frames) | (uintptr_t)a.frame_stride |
                             (uintptr_t)a.row_pitch) & 15u) == 0;
    const long long plane = (long long)a.H * a.W;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < units;
         u += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(u % chunks);
        const long long r = u / chunks;
        const int y = (int)(r % a.H);
        const int gi = (int)(r / a.H);
        const int g = a.g0 + gi;
        const int j0 = g * a.d;
        const int j1 = min(a.m, j0 + a.d);
        const int b0 = k * 16;
        const int nb = min(16, rowbytes - b0);
        const uint8_t *base = a.frames + (long long)y * a.row_pitch + b0;
        uint32_t tot[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) tot[i] = 0;
        if (aligned16 && nb == 16) {
            for (int jb = j0; jb < j1; jb += 256) {
                const int je = min(j1, jb + 256);
                uint32_t ev[4] = {0, 0, 0, 0}, od[4] = {0, 0, 0, 0};
                const uint8_t *p = base + (long long)jb * a.frame_stride;
                int j = jb;
#pragma unroll 4
                for (; j < je; ++j, p += a.frame_stride) {
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
                const uint8_t *p = base + (long long)j * a.frame_stride;
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (i < nb) tot[i] += p[i];
            }
        }
        const float fn = (float)(j1 - j0);
        float *o = a.out + (long long)gi * a.C * plane + (long long)y * a.W;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            if (i < nb) {
                const int ob = b0 + i;
                const int x = ob / a.C;
                const int c = ob - x * a.C;
                const float s = (float)tot[i];
                o[(long long)c * plane + x] = a.mean ? __fdiv_rn(s, fn) : s;
            }
        }
    }
}

cudaError_t launch_sda(const SdaArgs &a, int num_sms, cudaStream_t st) {
    const long long units = (long long)a.G * a.H * ((a.W * a.C + 15) / 16);
    long long blocks = (units + 255) / 256;
    const long long cap = (long long)num_sms * 8;  // 8 x 256 threads per SM, grid-stride beyond
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_sda_sum<<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace prnu
