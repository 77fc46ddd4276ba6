// prnu_static.cu -- allocation-free variant of prnu_denoise_residual.
//
// Some callers cannot allocate device memory at the time they need a residual:
// code running inside a CUDA stream capture (allocation is not a capturable
// operation), plug-ins whose host application owns all device allocations,
// or services that forbid allocation after start-up to keep their memory
// footprint fixed.  This entry point takes its scratch from a fixed
// file-scope device array instead of a caller-provided workspace, and calls no
// cudaMalloc, cudaFree or allocating library routine.
//
// The array lives in this translation unit's module: every GPU on which the
// module is loaded holds kStaticScratchBytes of device memory until the
// process exits.  All calls on a device share the one array, so calls whose
// GPU work overlaps in time (different streams or threads without ordering)
// race on it; calls ordered on one stream are safe.  Each call overwrites
// every scratch byte it reads before reading it, so nothing needs clearing
// between calls.
#include <cstdio>
#include <mutex>

#include "kernels.cuh"

namespace prnu {
int ctx_device(const prnu_ctx *ctx);
void **ctx_static_scratch(prnu_ctx *ctx);
prnu_status check_residual_request(const float *img, int H, int W, int C, const prnu_params *params,
                                   const float *residual_out, size_t *need);
prnu_status set_last_error(prnu_status s, const char *msg);
}  // namespace prnu

namespace {

constexpr size_t kStaticScratchBytes = 64ull << 20;  // 64 MiB

static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

std::mutex g_mu;

// Device address of g_scratch on the context's device, resolved once per
// context with that device current and kept in the context.  In host code the
// name g_scratch is only a host-side stand-in, never a device address, so
// kernels must receive this pointer.  Keeping it per context (rather than per
// process) means a context created after a device reset resolves the address
// of the re-loaded module instead of reusing a stale one.
cudaError_t scratch_of(prnu_ctx *ctx, void **out) {
    std::lock_guard<std::mutex> lk(g_mu);
    void **slot = prnu::ctx_static_scratch(ctx);
    if (!*slot) {
        const int dev = prnu::ctx_device(ctx);
        int prev = -1;
        cudaError_t e = cudaGetDevice(&prev);
        if (e != cudaSuccess) return e;
        if (prev != dev && (e = cudaSetDevice(dev)) != cudaSuccess) return e;
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (prev != dev) cudaSetDevice(prev);
        if (e != cudaSuccess) return e;
        *slot = p;
    }
    *out = *slot;
    return cudaSuccess;
}

}  // namespace

extern "C" prnu_status prnu_denoise_residual_static(prnu_ctx *ctx, const float *img, int H, int W, int C,
                                                    const prnu_params *params, float *residual_out, void *stream) {
    if (!ctx) return prnu::set_last_error(PRNU_EINVAL, "ctx is NULL");
    // the regular entry point's checks first: invalid input resolves nothing
    // (no module load) and launches nothing
    size_t need = 0;
    prnu_status s = prnu::check_residual_request(img, H, W, C, params, residual_out, &need);
    if (s != PRNU_OK) return s;
    if (need > kStaticScratchBytes) {
        char msg[320];
        snprintf(msg, sizeof msg,
                 "prnu_denoise_residual_static: a %d x %d x %d image with %s subbands needs %zu bytes of scratch, "
                 "more than the %zu-byte static scratch; use prnu_denoise_residual with a workspace",
                 H, W, C, params->dtype == PRNU_DTYPE_F32 ? "float32" : "16-bit", need, kStaticScratchBytes);
        return prnu::set_last_error(PRNU_ENOSPC, msg);
    }
    void *scratch = nullptr;
    const cudaError_t e = scratch_of(ctx, &scratch);
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof msg, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
        return prnu::set_last_error(PRNU_ECUDA, msg);
    }
    return prnu_denoise_residual(ctx, img, H, W, C, params, residual_out, scratch, kStaticScratchBytes, stream);
}
