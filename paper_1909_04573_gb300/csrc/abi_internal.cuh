// abi_internal.cuh -- host-side internals of libprnu shared by the
// translation units that implement prnu.h (context, error reporting, launch
// accounting, argument checks, workspace layouts, the denoise pipeline).
#pragma once

#include <cufft.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "kernels.cuh"

struct prnu_ctx {
    int device = 0;
    int sms = 0;
    double h64[prnu::kTaps];
    prnu::Filt filt;
    std::mutex mu;
    std::map<std::tuple<int, int, int, int>, cufftHandle> plans;  // (H, W, type, batch) -> plan
    std::map<std::tuple<int, int, int, int>, size_t> plan_work;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
    // per-kernel launch counters (always) and CUDA-event timing (opt-in)
    bool prof_on = false;
    std::vector<std::string> prof_sel;  // kernels to time (empty: all)
    std::vector<std::string> knames;
    std::vector<long long> klaunches;
    std::vector<double> kbytes;  // algorithmic bytes of the counted launches
    struct Rec {
        int kid;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    // autotuned level-1 analysis shape per (padded H, padded W, subband type)
    std::map<std::tuple<int, int, int>, int> tuned;
    // autotuned choices of the other launches per (padded H, padded W,
    // subband type, kind, level)
    std::map<std::tuple<int, int, int, int, int>, int> tuned_lv;
    // device address of the allocation-free entry point's scratch array,
    // resolved by that entry point's first call with this context
    void *static_scratch = nullptr;
};

namespace prnu {
namespace abi {

// Stores the message for prnu_last_error (thread-local) and returns s.
prnu_status fail(prnu_status s, const char *fmt, ...) __attribute__((format(printf, 2, 3)));

#define CU(call)                                                                                      \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return fail(PRNU_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define CUFFT(call)                                                                                   \
    do {                                                                                              \
        cufftResult r_ = (call);                                                                      \
        if (r_ != CUFFT_SUCCESS) return fail(PRNU_ECUDA, "%s: cufft error %d", #call, (int)r_);      \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Brackets one kernel (or library call) with CUDA events on its stream when
// profiling is on; always counts the launch.
struct Launch {
    prnu_ctx *ctx;
    cudaStream_t st;
    int kid = -1;
    cudaEvent_t a = nullptr, b = nullptr;
    Launch(prnu_ctx *c, const char *name, cudaStream_t s, int kernels = 1, double bytes = 0.0) : ctx(c), st(s) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (size_t i = 0; i < ctx->knames.size(); ++i)
            if (ctx->knames[i] == name) kid = (int)i;
        if (kid < 0) {
            kid = (int)ctx->knames.size();
            ctx->knames.push_back(name);
            ctx->klaunches.push_back(0);
            ctx->kbytes.push_back(0.0);
        }
        ctx->klaunches[kid] += kernels;
        ctx->kbytes[kid] += bytes;
        bool timed = ctx->prof_on && ctx->prof_sel.empty();
        for (size_t i = 0; ctx->prof_on && !timed && i < ctx->prof_sel.size(); ++i) timed = ctx->prof_sel[i] == name;
        if (timed) {
            a = take();
            b = take();
            if (a && b) record(a);
        }
    }
    cudaEvent_t take() {
        if (!ctx->pool.empty()) {
            cudaEvent_t e = ctx->pool.back();
            ctx->pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        return cudaEventCreate(&e) == cudaSuccess ? e : nullptr;
    }
    // Under stream capture the record becomes an event node of the graph, so
    // that each replay re-times the launch; the events stay checked out of the
    // pool until prnu_profile_reset.
    void record(cudaEvent_t e) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
            cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
        else
            cudaEventRecord(e, st);
    }
    ~Launch() {
        if (a && b) {
            record(b);
            std::lock_guard<std::mutex> lk(ctx->mu);
            ctx->recs.push_back({kid, a, b});
        }
    }
};

inline cudaStream_t S(void *p) { return reinterpret_cast<cudaStream_t>(p); }

prnu_status check_geometry(int H, int W, int C);
// Validates params against the geometry; fills `win` (nullable).
prnu_status check_params(const prnu_params *p, int H, int W, Win *win);
prnu_status check_ws(void *ws, size_t ws_bytes, size_t need);
// Frames of an accumulate call (element size fes bytes: 1 uint8, 2 float16).
prnu_status check_frames(const uint8_t *frames, int m, int H, int W, int C, size_t frame_stride, size_t row_pitch,
                         int d, int fes = 1);

inline int padded(int n, int levels) {
    const int m = 1 << levels;
    return (n + m - 1) / m * m;
}

// Workspace of the denoise pipeline over P planes of one geometry.
struct Layout {
    size_t X = 0;  // group sums [P][H][W] (accumulate only)
    size_t LLh[kMaxLevels + 1] = {}, LLl[kMaxLevels + 1] = {}, Rn[kMaxLevels + 1] = {};
    size_t D[kMaxLevels + 1] = {}, N[kMaxLevels + 1] = {};
    size_t end = 0;
};

constexpr size_t kAlign = 256;
Layout make_layout(int H, int W, long long P, int L, bool withX, int sdt = SB_F32);

// Analysis, shrink and synthesis of P planes; the level-1 step (residual or
// MLE) is described by `fin`, whose coefficient pointers are filled here.
// With `ckpt` (the forward's detail coefficients of all levels, float32, level
// after level, each [3][P][Hp/2^l][Wp/2^l]) the shrink is replaced by its
// adjoint: `in` is then a residual gradient and the result (accumulated into
// fin.res_out) the gradient of the input; dL/dsigma0 is added to *g_sigma.
// run_denoise phases: everything; analysis, shrink and synthesis down to
// level 2 only; the level-1 synthesis (and its epilogue) only, from subbands a
// kDenoiseUpToLevel2 call left in the same workspace; everything but the
// level-1 analysis, whose outputs the fused group-sum kernel left in the layout.
constexpr int kDenoiseAll = 0, kDenoiseUpToLevel2 = 1, kDenoiseLevel1 = 2, kDenoiseAfterL1Analysis = 3;
// Arguments of the level-l analysis of P planes of the layout lo in ws.
AnaArgs analysis_args(const prnu_ctx *ctx, const float *in, int H, int W, int P, const prnu_params &prm,
                      PlaneScale sc, int scale_on, char *ws, const Layout &lo, int l);
prnu_status run_denoise(prnu_ctx *ctx, const float *in, int H, int W, int P, const prnu_params &prm, const Win &win,
                        PlaneScale sc, int scale_on, char *ws, const Layout &lo, FinalArgs fin, bool mle,
                        cudaStream_t st, const float *ckpt = nullptr, double *g_sigma = nullptr,
                        int phase = kDenoiseAll);

// cuFFT plan cache: (H, W, type, batch) -> plan without an auto-allocated
// work area; batched planes are contiguous with the default distances.
prnu_status get_plan(prnu_ctx *ctx, int H, int W, cufftType type, int batch, cufftHandle *plan, size_t *work);

constexpr int kRedBlocks = 512;
constexpr int kPipeSdaBlocks = 6;  // SDA sums blocks per SM beside a pipelined accumulate's denoising

// Workspace of finalize (one plane at a time) and of a PCE batch of n queries.
struct FftLayout {
    size_t cplx = 0;                  // complex: max(2n half spectra, one full plane)
    size_t real = 0;                  // float: 2n planes (X_i, Y_i) or (M, Mn)
    size_t colmean = 0, rowmean = 0;  // doubles
    size_t colpart = 0;               // doubles: partial column sums per 64-row band
    size_t part = 0, tmp = 0, mom0 = 0;
    size_t pm = 0, pe = 0, pv = 0, pi = 0, scal = 0;
    size_t tw = 0, c0 = 0;            // own-FFT correlation: twiddles, C(0, 0) per query
    bool own_fft = false;             // PCE correlation by k_corr.cu instead of cuFFT
    size_t work = 0, end = 0;
    int nb = 0, nbm = 0;              // reduction blocks per query
};
prnu_status fft_layout(prnu_ctx *ctx, int H, int W, int n, FftLayout *out);

}  // namespace abi
}  // namespace prnu
