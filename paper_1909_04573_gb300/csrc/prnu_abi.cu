// prnu_abi.cu -- host side of libprnu: context, filter bank, argument
// validation, workspace layout and the extern "C" entry points of prnu.h.
#include <cufft.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "abi_internal.cuh"

using namespace prnu;
using namespace prnu::abi;

namespace prnu {
namespace abi {

thread_local std::string tl_err;

prnu_status fail(prnu_status s, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
prnu_status fail(prnu_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    tl_err = buf;
    return s;
}




// ---------------------------------------------------------------------------
// Filter bank.  The 8-tap orthonormal Daubechies lowpass (4 vanishing
// moments) is the solution of eight equations:
//   sum_k h_k h_{k+2n} = delta_n        (n = 0..3, double-shift orthonormality)
//   sum_k (-1)^k k^q h_k = 0            (q = 0..3, vanishing moments of g)
// solved here by Newton's method in double precision, started from the
// minimum-phase solution rounded to 4 decimals (Daubechies' published table),
// which selects that solution among the equations' roots.
// ---------------------------------------------------------------------------
bool derive_filter(double h[kTaps]) {
    const double init[kTaps] = {0.2304, 0.7148, 0.6309, -0.0280, -0.1870, 0.0308, 0.0329, -0.0106};
    for (int k = 0; k < kTaps; ++k) h[k] = init[k];
    for (int it = 0; it < 30; ++it) {
        double F[kTaps], J[kTaps][kTaps];
        for (int n = 0; n < 4; ++n) {
            double s = 0.0;
            for (int k = 0; k + 2 * n < kTaps; ++k) s += h[k] * h[k + 2 * n];
            F[n] = s - (n == 0 ? 1.0 : 0.0);
            for (int m = 0; m < kTaps; ++m) {
                double d = 0.0;
                if (m + 2 * n < kTaps) d += h[m + 2 * n];
                if (m - 2 * n >= 0) d += h[m - 2 * n];
                J[n][m] = d;
            }
        }
        for (int q = 0; q < 4; ++q) {
            double s = 0.0;
            for (int k = 0; k < kTaps; ++k) {
                const double c = (k % 2 ? -1.0 : 1.0) * std::pow((double)k, q);
                s += c * h[k];
                J[4 + q][k] = c;
            }
            F[4 + q] = s;
        }
        // solve J dx = F (Gaussian elimination, partial pivoting)
        double A[kTaps][kTaps + 1];
        for (int i = 0; i < kTaps; ++i) {
            for (int j = 0; j < kTaps; ++j) A[i][j] = J[i][j];
            A[i][kTaps] = F[i];
        }
        for (int c = 0; c < kTaps; ++c) {
            int piv = c;
            for (int r = c + 1; r < kTaps; ++r)
                if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
            if (std::fabs(A[piv][c]) < 1e-300) return false;
            if (piv != c)
                for (int j = 0; j <= kTaps; ++j) std::swap(A[c][j], A[piv][j]);
            for (int r = c + 1; r < kTaps; ++r) {
                const double f = A[r][c] / A[c][c];
                for (int j = c; j <= kTaps; ++j) A[r][j] -= f * A[c][j];
            }
        }
        double dx[kTaps];
        for (int r = kTaps - 1; r >= 0; --r) {
            double s = A[r][kTaps];
            for (int j = r + 1; j < kTaps; ++j) s -= A[r][j] * dx[j];
            dx[r] = s / A[r][r];
        }
        for (int k = 0; k < kTaps; ++k) h[k] -= dx[k];
    }
    // verify: equations, normalisation sum h = sqrt(2), minimum-phase ordering
    double sum = 0.0, worst = 0.0;
    for (int k = 0; k < kTaps; ++k) sum += h[k];
    for (int n = 0; n < 4; ++n) {
        double s = 0.0;
        for (int k = 0; k + 2 * n < kTaps; ++k) s += h[k] * h[k + 2 * n];
        worst = std::fmax(worst, std::fabs(s - (n == 0 ? 1.0 : 0.0)));
    }
    for (int q = 0; q < 4; ++q) {
        double s = 0.0;
        for (int k = 0; k < kTaps; ++k) s += (k % 2 ? -1.0 : 1.0) * std::pow((double)k, q) * h[k];
        worst = std::fmax(worst, std::fabs(s) / std::pow(7.0, q));
    }
    return worst < 1e-13 && std::fabs(sum - std::sqrt(2.0)) < 1e-12 && h[0] > 0.2 && h[1] > h[0];
}

prnu_status check_geometry(int H, int W, int C) {
    if (H < 16 || W < 16 || H > 16384 || W > 16384) return fail(PRNU_EINVAL, "H, W must be in [16, 16384] (got %d x %d)", H, W);
    if (C != 1 && C != 3) return fail(PRNU_EINVAL, "C must be 1 or 3 (got %d)", C);
    return PRNU_OK;
}

prnu_status check_params(const prnu_params *p, int H, int W, Win *win) {
    if (!p) return fail(PRNU_EINVAL, "params is NULL");
    if (p->levels < 1 || p->levels > kMaxLevels) return fail(PRNU_EINVAL, "levels must be in [1, %d]", kMaxLevels);
    if (H < (1 << p->levels) || W < (1 << p->levels)) return fail(PRNU_EINVAL, "H, W must be >= 2^levels");
    if (!(p->sigma0 >= 0.f) || !std::isfinite(p->sigma0)) return fail(PRNU_EINVAL, "sigma0 must be finite and >= 0");
    if (p->n_windows < 1 || p->n_windows > 4) return fail(PRNU_EINVAL, "n_windows must be in [1, 4]");
    if (p->pad_mode != 0) return fail(PRNU_EUNSUPPORTED, "pad_mode %d not supported (0 = mirror)", p->pad_mode);
    if (p->dtype < PRNU_DTYPE_F32 || p->dtype > PRNU_DTYPE_BF16)
        return fail(PRNU_EINVAL, "dtype %d invalid (0 = float32, 1 = float16, 2 = bfloat16 subbands)", p->dtype);
    if (p->frame_dtype != PRNU_FRAMES_U8 && p->frame_dtype != PRNU_FRAMES_F16)
        return fail(PRNU_EINVAL, "frame_dtype %d invalid (0 = uint8, 1 = float16)", p->frame_dtype);
    if (p->compensated != 0 && p->compensated != 1) return fail(PRNU_EINVAL, "compensated must be 0 or 1");
    if (p->sda_blocks_per_sm < 0 || p->sda_blocks_per_sm > 32)
        return fail(PRNU_EINVAL, "sda_blocks_per_sm must be in 0..32");
    if (p->pipeline_passes < 0 || p->pipeline_passes > 64)
        return fail(PRNU_EINVAL, "pipeline_passes must be in 0..64");
    if (p->sda_fusion < PRNU_SDA_FUSED || p->sda_fusion > 256)
        return fail(PRNU_EINVAL, "sda_fusion must be PRNU_SDA_FUSED (-2), PRNU_SDA_SEPARATE (-1), 0 or a strip "
                                 "count in 1..256");
    if (win) {
        win->n = p->n_windows;
        for (int i = 0; i < 4; ++i) {
            win->r[i] = 0;
            win->inv[i] = 1.f;
        }
        for (int i = 0; i < p->n_windows; ++i) {
            const int w = p->windows[i];
            if (w < 1 || w > 2 * kMaxRadius + 1 || w % 2 == 0) return fail(PRNU_EINVAL, "windows must be odd in [1, 9]");
            win->r[i] = w / 2;
            win->inv[i] = (float)(1.0 / ((double)w * w));
        }
    }
    return PRNU_OK;
}



Layout make_layout(int H, int W, long long P, int L, bool withX, int sdt) {
    Layout lo;
    const size_t es = subband_bytes(sdt);  // detail, noise and noise-LL storage
    const long long Hp = padded(H, L), Wp = padded(W, L);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, kAlign);
        return o;
    };
    if (withX) lo.X = take((size_t)P * H * W * sizeof(float));
    for (int l = 1; l <= L; ++l) {
        const size_t A = (size_t)(Hp >> l) * (size_t)(Wp >> l);
        if (l < L) {
            lo.LLh[l] = take(P * A * sizeof(float));
            lo.LLl[l] = take(P * A * sizeof(float));
            lo.Rn[l] = take(P * A * es);
        }
        lo.D[l] = take(3 * P * A * es);
        lo.N[l] = take(3 * P * A * es);
    }
    lo.end = off;
    return lo;
}

// Arguments of the level-l analysis of P planes of the layout lo in ws
// (level 1 reads `in`).
AnaArgs analysis_args(const prnu_ctx *ctx, const float *in, int H, int W, int P, const prnu_params &prm,
                      PlaneScale sc, int scale_on, char *ws, const Layout &lo, int l) {
    const int L = prm.levels;
    const int Hp = padded(H, L), Wp = padded(W, L);
    auto F = [&](size_t off) { return reinterpret_cast<float *>(ws + off); };
    const long long A = (long long)(Hp >> l) * (Wp >> l);
    const size_t es = subband_bytes(prm.dtype);
    auto SB = [&](size_t off, int k) { return static_cast<void *>(ws + off + (size_t)k * P * A * es); };
    AnaArgs a{};
    a.inh = l == 1 ? in : F(lo.LLh[l - 1]);
    a.inl = l == 1 ? nullptr : F(lo.LLl[l - 1]);
    a.R = Hp >> (l - 1);
    a.Cc = Wp >> (l - 1);
    a.H = H;
    a.W = W;
    a.P = P;
    a.LLh = l < L ? F(lo.LLh[l]) : nullptr;
    a.LLl = l < L ? F(lo.LLl[l]) : nullptr;
    a.LH = SB(lo.D[l], 0);
    a.HL = SB(lo.D[l], 1);
    a.HH = SB(lo.D[l], 2);
    a.sdt = prm.dtype;
    a.sc = sc;
    a.scale_on = scale_on;
    a.f = ctx->filt;
    return a;
}

// Analysis, shrink and synthesis of P planes; the level-1 step (residual or
// MLE) is described by `fin`, whose coefficient pointers are filled here.
// Phase kDenoiseAfterL1Analysis starts at the level-1 shrink: the level-1
// analysis outputs are already in the layout (the fused group-sum kernel).
prnu_status run_denoise(prnu_ctx *ctx, const float *in, int H, int W, int P, const prnu_params &prm, const Win &win,
                        PlaneScale sc, int scale_on, char *ws, const Layout &lo, FinalArgs fin, bool mle,
                        cudaStream_t st, const float *ckpt, double *g_sigma, int phase) {
    size_t ckpt_off = 0;  // floats of the levels before l in the checkpoint
    const int L = prm.levels;
    const int Hp = padded(H, L), Wp = padded(W, L);
    const int sdt = prm.dtype;
    const size_t es = subband_bytes(sdt);
    // typed subband k of a region holding 3 (or 1) planes groups of P planes
    auto SB = [&](size_t off, long long A, int k) { return static_cast<void *>(ws + off + (size_t)k * P * A * es); };
    // the tuner's choice for a launch kind at level l (0: the default rule)
    auto choice = [&](int kind, int l) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        auto it = ctx->tuned_lv.find(std::make_tuple(Hp, Wp, sdt, kind, l));
        return it == ctx->tuned_lv.end() ? 0 : it->second;
    };
    for (int l = 1; l <= L && phase != kDenoiseLevel1; ++l) {
        const long long A = (long long)(Hp >> l) * (Wp >> l);
        const AnaArgs a = analysis_args(ctx, in, H, W, P, prm, sc, scale_on, ws, lo, l);
        if (!(l == 1 && phase == kDenoiseAfterL1Analysis)) {
            const double in_b = l == 1 ? (double)P * H * W * 4 : (double)P * a.R * a.Cc * 8;
            const double out_b = (double)P * A * (3.0 * es + (l < L ? 8 : 0));
            Launch t(ctx, l == 1 ? "analysis_l1" : "analysis", st, 1, in_b + out_b);
            int shape = kStreamShapeDefault;
            if (l == 1) {
                std::lock_guard<std::mutex> lk(ctx->mu);
                auto it = ctx->tuned.find(std::make_tuple(Hp, Wp, sdt));
                if (it != ctx->tuned.end()) shape = it->second;
            } else {
                shape = choice(kTuneAnalysis, l);
            }
            CU(launch_analysis(a, l == 1, st, shape));
        }
        if (ckpt) {  // adjoint: D holds the gradient of the noise coefficients
            ShrinkBwdArgs b{};
            b.c = ckpt + ckpt_off;
            b.gn = static_cast<const float *>(SB(lo.D[l], A, 0));
            b.gc = static_cast<float *>(SB(lo.N[l], A, 0));
            b.R = Hp >> l;
            b.Cc = Wp >> l;
            b.nplanes = 3 * P;
            b.s2 = prm.sigma0 * prm.sigma0;
            b.two_sigma0 = 2.f * prm.sigma0;
            b.win = win;
            b.g_sigma = g_sigma;
            ckpt_off += (size_t)3 * P * A;
            Launch t(ctx, "shrink_bwd", st, 1, 3.0 * b.nplanes * b.R * b.Cc * 4);
            CU(launch_shrink_bwd(b, st));
            continue;
        }
        ShrinkArgs s{};
        s.in = SB(lo.D[l], A, 0);
        s.out = SB(lo.N[l], A, 0);
        s.sdt = sdt;
        s.R = Hp >> l;
        s.Cc = Wp >> l;
        s.nplanes = 3 * P;
        s.s2 = prm.sigma0 * prm.sigma0;
        s.s2_dev = nullptr;
        s.win = win;
        {
            Launch t(ctx, "shrink", st, 1, 2.0 * s.nplanes * s.R * s.Cc * es);
            CU(launch_shrink(s, st, choice(kTuneShrink, l)));
        }
    }
    // PCE mode with three channels: the synthesis is linear, so levels L..1
    // synthesise the grey combination of the channels' noise, one plane per image
    const bool grey = fin.pce && fin.C == 3;
    const int Ps = grey ? P / 3 : P;
    for (int l = L; l >= 2 && phase != kDenoiseLevel1; --l) {
        const long long A = (long long)(Hp >> l) * (Wp >> l);
        SynArgs y{};
        y.LL = l == L ? nullptr : SB(lo.Rn[l], A, 0);
        y.LH = SB(lo.N[l], A, 0);
        y.HL = SB(lo.N[l], A, 1);
        y.HH = SB(lo.N[l], A, 2);
        y.sdt = sdt;
        y.Rc = Hp >> l;
        y.Cc = Wp >> l;
        y.P = Ps;
        y.gray3 = grey;
        y.out = SB(lo.Rn[l - 1], 0, 0);
        y.f = ctx->filt;
        {
            Launch t(ctx, "synthesis", st, 1, (double)P * A * es * 3 + (double)Ps * A * es * (y.LL ? 5 : 4));
            CU(launch_synthesis(y, st, choice(kTuneSynthesis, l)));
        }
    }
    if (phase == kDenoiseUpToLevel2) return PRNU_OK;
    const long long A1 = (long long)(Hp >> 1) * (Wp >> 1);
    fin.LL = L == 1 ? nullptr : SB(lo.Rn[1], A1, 0);
    fin.LH = SB(lo.N[1], A1, 0);
    fin.HL = SB(lo.N[1], A1, 1);
    fin.HH = SB(lo.N[1], A1, 2);
    fin.sdt = sdt;
    fin.compensated = prm.compensated;
    fin.Rc = Hp >> 1;
    fin.Cc = Wp >> 1;
    fin.H = H;
    fin.W = W;
    fin.f = ctx->filt;
    {
        const double cin = (double)P * A1 * es * 3 + (fin.LL ? (double)Ps * A1 * es : 0.0);
        const double io = mle ? (double)P * H * W * 4 + (double)fin.C * H * W * 16 * (prm.compensated ? 2 : 1)
                        : fin.pce ? (double)fin.G * H * W * 4 * (fin.C + 3)
                                  : (double)P * H * W * 4 * (fin.accumulate ? 2 : 1);
        Launch t(ctx, mle ? "final_mle" : fin.pce ? "final_pce" : "final_residual", st, 1, cin + io);
        CU(launch_final(fin, mle, st, mle ? choice(kTuneFinal, 1) : 0));
    }
    return PRNU_OK;
}

prnu_status check_ws(void *ws, size_t ws_bytes, size_t need) {
    if (need > ws_bytes) return fail(PRNU_ENOSPC, "workspace too small: need %zu bytes, got %zu", need, ws_bytes);
    if (need > 0 && (reinterpret_cast<uintptr_t>(ws) % kAlign)) return fail(PRNU_EINVAL, "workspace must be 256-byte aligned");
    return PRNU_OK;
}

prnu_status check_frames(const uint8_t *frames, int m, int H, int W, int C, size_t frame_stride, size_t row_pitch,
                         int d, int fes) {
    if (!frames) return fail(PRNU_EINVAL, "frames is NULL");
    if (m < 1) return fail(PRNU_EINVAL, "m must be >= 1");
    if (d < 1 || d > m) return fail(PRNU_EINVAL, "d must be in [1, m] (d=%d, m=%d)", d, m);
    if (d > 65793) return fail(PRNU_EINVAL, "d must be <= 65793 (exact float32 group sums)");
    if (row_pitch < (size_t)W * C * fes) return fail(PRNU_EINVAL, "row_pitch < W*C*element size");
    if (m > 1 && frame_stride < (size_t)(H - 1) * row_pitch + (size_t)W * C * fes)
        return fail(PRNU_EINVAL, "frame_stride too small");
    if (fes == 2 && ((reinterpret_cast<uintptr_t>(frames) | frame_stride | row_pitch) & 1u))
        return fail(PRNU_EINVAL, "float16 frames need 2-byte aligned pointer and strides");
    return PRNU_OK;
}

// cuFFT plan cache: (H, W, type, batch) -> plan without an auto-allocated
// work area; batched planes are contiguous with the default distances.
prnu_status get_plan(prnu_ctx *ctx, int H, int W, cufftType type, int batch, cufftHandle *plan, size_t *work) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    const auto key = std::make_tuple(H, W, (int)type, batch);
    auto it = ctx->plans.find(key);
    if (it == ctx->plans.end()) {
        cufftHandle p;
        CUFFT(cufftCreate(&p));
        CUFFT(cufftSetAutoAllocation(p, 0));
        size_t ws = 0;
        int dims[2] = {H, W};
        cufftResult r = cufftMakePlanMany(p, 2, dims, nullptr, 1, 0, nullptr, 1, 0, type, batch, &ws);
        if (r != CUFFT_SUCCESS) {
            cufftDestroy(p);
            return fail(PRNU_ECUDA, "cufftMakePlanMany(%d x %d, batch %d) failed: %d", H, W, batch, (int)r);
        }
        ctx->plans[key] = p;
        ctx->plan_work[key] = ws;
        it = ctx->plans.find(key);
    }
    *plan = it->second;
    *work = ctx->plan_work[key];
    return PRNU_OK;
}



prnu_status fft_layout(prnu_ctx *ctx, int H, int W, int n, FftLayout *out) {
    FftLayout f;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, kAlign);
        return o;
    };
    const size_t hw = (size_t)H * W;
    const size_t nh = (size_t)H * (W / 2 + 1);
    f.nb = (int)std::min<size_t>(256, std::max<size_t>(1, hw / (256 * 16)));
    f.nbm = f.nb;
    f.own_fft = corr_fft_supported(H, W);
    const size_t nh_pce = f.own_fft ? (size_t)H * corr_pitch(W) : nh;  // padded rows for the own FFT
    f.cplx = take(2 * (size_t)std::max(n, 1) * std::max(nh, nh_pce) * sizeof(cufftComplex));
    f.real = take(2 * (size_t)std::max(n, 1) * hw * sizeof(float));
    f.colmean = take((size_t)W * sizeof(double));
    f.colpart = take((size_t)((H + 63) / 64) * W * sizeof(double));
    f.rowmean = take((size_t)H * sizeof(double));
    f.part = take((size_t)kRedBlocks * 2 * sizeof(double));
    f.tmp = take(2 * sizeof(double));
    f.mom0 = take(2 * sizeof(double));
    f.pm = take((size_t)n * f.nbm * 4 * sizeof(double));
    f.pe = take((size_t)n * f.nb * sizeof(double));
    f.pv = take((size_t)n * f.nb * sizeof(float));
    f.pi = take((size_t)n * f.nb * sizeof(long long));
    f.scal = take((size_t)n * pce_scalars_bytes());
    f.tw = take(f.own_fft ? corr_twiddle_count(H, W) * sizeof(float2) : 0);
    f.c0 = take((size_t)std::max(n, 1) * sizeof(float));
    size_t w = 0, wmax = 0;
    cufftHandle p;
    prnu_status s;
    if ((s = get_plan(ctx, H, W, CUFFT_R2C, 1, &p, &w)) != PRNU_OK) return s;  // finalize's Wiener step
    wmax = std::max(wmax, w);
    if ((s = get_plan(ctx, H, W, CUFFT_C2R, 1, &p, &w)) != PRNU_OK) return s;
    wmax = std::max(wmax, w);
    if (!f.own_fft) {  // batched plans of the PCE correlation
        if ((s = get_plan(ctx, H, W, CUFFT_R2C, 2 * n, &p, &w)) != PRNU_OK) return s;
        wmax = std::max(wmax, w);
        if ((s = get_plan(ctx, H, W, CUFFT_C2R, n, &p, &w)) != PRNU_OK) return s;
        wmax = std::max(wmax, w);
    }
    f.work = take(wmax);
    f.end = off;
    *out = f;
    return PRNU_OK;
}


// Group-sum arguments of groups g0 .. g0+G-1 of `frames` into X.
SdaArgs sda_args(const uint8_t *frames, int m, int H, int W, int C, size_t fs, size_t rp, int d, int g0, int G,
                 const prnu_params &prm, float *X, int blocks_per_sm) {
    SdaArgs sa{};
    sa.frames = frames;
    sa.frame_stride = (long long)fs;
    sa.row_pitch = (long long)rp;
    sa.m = m;
    sa.H = H;
    sa.W = W;
    sa.C = C;
    sa.d = d;
    sa.g0 = g0;
    sa.G = G;
    sa.out = X;
    sa.mean = 0;
    sa.frame_half = prm.frame_dtype == PRNU_FRAMES_F16;
    sa.blocks_per_sm = blocks_per_sm > 0 ? blocks_per_sm : prm.sda_blocks_per_sm;
    return sa;
}

// Frame bytes the groups g0 .. g0+G-1 read.
double group_frame_bytes(int m, int H, int W, int C, int d, int g0, int G, const prnu_params &prm) {
    return (double)(std::min(m, (g0 + G) * d) - g0 * d) * H * W * C * (prm.frame_dtype == PRNU_FRAMES_F16 ? 2 : 1);
}

// Group sums of groups g0 .. g0+G-1 of `frames` into the pass layout's X.
prnu_status sda_pass(prnu_ctx *ctx, const uint8_t *frames, int m, int H, int W, int C, size_t fs, size_t rp, int d,
                     int g0, int G, const prnu_params &prm, char *ws, cudaStream_t st, int blocks_per_sm = 0) {
    const int P = G * C;
    const Layout lo = make_layout(H, W, P, prm.levels, true, prm.dtype);
    const SdaArgs sa = sda_args(frames, m, H, W, C, fs, rp, d, g0, G, prm, reinterpret_cast<float *>(ws + lo.X),
                                blocks_per_sm);
    const double fr = group_frame_bytes(m, H, W, C, d, g0, G, prm);
    Launch t(ctx, "sda_sum", st, 1, fr + (double)P * H * W * 4);
    CU(launch_sda(sa, ctx->sms, st));
    return PRNU_OK;
}

// Denoise + MLE of the G group sums in the pass layout's X into num/den.
prnu_status denoise_pass(prnu_ctx *ctx, int m, int H, int W, int C, int d, int g0, int G, const prnu_params &prm,
                         const Win &win, float *num, float *den, char *ws, cudaStream_t st,
                         int phase = kDenoiseAll) {
    const int P = G * C;
    const Layout lo = make_layout(H, W, P, prm.levels, true, prm.dtype);
    const PlaneScale sc{d, m, g0, C, nullptr};
    FinalArgs fin{};
    fin.C = C;
    fin.G = G;
    fin.X = reinterpret_cast<const float *>(ws + lo.X);
    fin.sc = sc;
    fin.num = num;
    fin.den = den;
    return run_denoise(ctx, reinterpret_cast<const float *>(ws + lo.X), H, W, P, prm, win, sc, 1, ws, lo, fin, true, st,
                       nullptr, nullptr, phase);
}

// Process groups g0 .. g0+G-1 of `frames` into num/den.  Frames in device
// memory (fuse_ok) take the fused group-sum + level-1 analysis kernel where it
// applies: by default for groups of at least kFuseMinGroup frames (shorter
// groups leave the fused kernel's per-stage hand-off and analysis too little
// summing to hide behind; measured), always with PRNU_SDA_FUSED or a strip
// count, never with PRNU_SDA_SEPARATE.
constexpr int kFuseMinGroup = 16;
prnu_status accumulate_pass(prnu_ctx *ctx, const uint8_t *frames, int m, int H, int W, int C, size_t fs, size_t rp,
                            int d, int g0, int G, const prnu_params &prm, const Win &win, float *num, float *den,
                            char *ws, cudaStream_t st, bool fuse_ok = true) {
    if (fuse_ok && (prm.sda_fusion >= 1 || prm.sda_fusion == PRNU_SDA_FUSED ||
                    (prm.sda_fusion == 0 && d >= kFuseMinGroup))) {
        const int P = G * C;
        const Layout lo = make_layout(H, W, P, prm.levels, true, prm.dtype);
        float *X = reinterpret_cast<float *>(ws + lo.X);
        const SdaArgs sa = sda_args(frames, m, H, W, C, fs, rp, d, g0, G, prm, X, 0);
        const AnaArgs a = analysis_args(ctx, X, H, W, P, prm, PlaneScale{d, m, g0, C, nullptr}, 1, ws, lo, 1);
        if (sda_dwt_applies(sa, a, nullptr)) {
            {
                const double l1 = (double)P * (a.R / 2) * (a.Cc / 2) * (3.0 * subband_bytes(prm.dtype) +
                                                                      (prm.levels > 1 ? 8 : 0));
                Launch t(ctx, "sda_dwt", st, 1, group_frame_bytes(m, H, W, C, d, g0, G, prm) + (double)P * H * W * 4 + l1);
                CU(launch_sda_dwt(sa, a, nullptr, ctx->sms, st, prm.sda_fusion > 0 ? prm.sda_fusion : 0));
            }
            return denoise_pass(ctx, m, H, W, C, d, g0, G, prm, win, num, den, ws, st, kDenoiseAfterL1Analysis);
        }
    }
    prnu_status s = sda_pass(ctx, frames, m, H, W, C, fs, rp, d, g0, G, prm, ws, st);
    if (s != PRNU_OK) return s;
    return denoise_pass(ctx, m, H, W, C, d, g0, G, prm, win, num, den, ws, st);
}

// Passes of Gp2 groups through two pass layouts in ws: the group sums of
// pass k+1 run on the context's side stream (at most sda_bps blocks per SM)
// while pass k is denoised on st; events hand each layout back and forth.
// Under stream capture the side stream joins the capture through the events.
prnu_status accumulate_pipelined(prnu_ctx *ctx, const uint8_t *frames, int m, int H, int W, int C, size_t fs,
                                 size_t rp, int d, int g, int Gp2, const prnu_params &prm, const Win &win, float *num,
                                 float *den, char *ws, int sda_bps, cudaStream_t st) {
    prnu_status s;
    const size_t half = align_up(make_layout(H, W, (long long)Gp2 * C, prm.levels, true, prm.dtype).end, kAlign);
    char *wsb[2] = {ws, ws + half};
    cudaStream_t side = ctx->copy_stream;
    for (int b = 0; b < 2; ++b) CU(cudaEventRecord(ctx->ev_free[b], st));  // after prior work on st
    int k = 0;
    for (int g0 = 0; g0 < g; g0 += Gp2, ++k) {
        const int G = std::min(Gp2, g - g0), b = k & 1;
        CU(cudaStreamWaitEvent(side, ctx->ev_free[b], 0));
        if ((s = sda_pass(ctx, frames, m, H, W, C, fs, rp, d, g0, G, prm, wsb[b], side, sda_bps)) != PRNU_OK) return s;
        CU(cudaEventRecord(ctx->ev_copied[b], side));
        CU(cudaStreamWaitEvent(st, ctx->ev_copied[b], 0));
        if ((s = denoise_pass(ctx, m, H, W, C, d, g0, G, prm, win, num, den, wsb[b], st)) != PRNU_OK) return s;
        CU(cudaEventRecord(ctx->ev_free[b], st));
    }
    return PRNU_OK;
}

// Largest number of groups per pass whose layout fits in `bytes`.
int groups_fitting(int H, int W, int C, int L, size_t bytes, int gmax, int sdt) {
    int lo = 0, hi = gmax;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (make_layout(H, W, (long long)mid * C, L, true, sdt).end <= bytes)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

}  // namespace abi
}  // namespace prnu

namespace {

// One pass over G groups of several cameras of one geometry: the group and
// camera table goes to the device through one small kernel (by value, so the
// sequence stays capturable in a CUDA graph), then the usual kernels run with
// per-group frame pointers, counts and camera routing.
prnu_status accumulate_pass_multi(prnu_ctx *ctx, const PassDesc &pd, int H, int W, int C, const prnu_params &prm,
                                  const Win &win, char *ws, cudaStream_t st) {
    const int G = pd.G, P = G * C;
    const Layout lo = make_layout(H, W, P, prm.levels, true, prm.dtype);
    PassDesc *dpd = reinterpret_cast<PassDesc *>(ws + lo.end);
    {
        Launch t(ctx, "put_desc", st, 1, 0.0);
        CU(launch_put_desc(pd, dpd, st));
    }
    SdaArgs sa{};
    sa.H = H;
    sa.W = W;
    sa.C = C;
    sa.G = G;
    sa.out = reinterpret_cast<float *>(ws + lo.X);
    sa.mean = 0;
    sa.frame_half = prm.frame_dtype == PRNU_FRAMES_F16;
    sa.gd = dpd->g;
    const PlaneScale sc{1, 1, 0, C, dpd->g};
    long long nfr = 0;  // frames of the pass
    for (int i = 0; i < G; ++i) nfr += pd.g[i].n;
    const double fr = (double)nfr * H * W * C * (sa.frame_half ? 2 : 1);  // their bytes
    // the group sums with the level-1 analysis in one kernel where it applies:
    // by default when the pass's groups average kFuseMinGroup frames or more
    const AnaArgs a1 = analysis_args(ctx, sa.out, H, W, P, prm, sc, 1, ws, lo, 1);
    const bool want = prm.sda_fusion >= 1 || prm.sda_fusion == PRNU_SDA_FUSED ||
                      (prm.sda_fusion == 0 && nfr >= (long long)kFuseMinGroup * G);
    const bool fused = want && sda_dwt_applies(sa, a1, &pd);
    if (fused) {
        const double l1 = (double)P * (a1.R / 2) * (a1.Cc / 2) * (3.0 * subband_bytes(prm.dtype) +
                                                                (prm.levels > 1 ? 8 : 0));
        Launch t(ctx, "sda_dwt", st, 1, fr + (double)P * H * W * 4 + l1);
        CU(launch_sda_dwt(sa, a1, &pd, ctx->sms, st, prm.sda_fusion > 0 ? prm.sda_fusion : 0));
    } else {
        Launch t(ctx, "sda_sum", st, 1, fr + (double)P * H * W * 4);
        CU(launch_sda(sa, ctx->sms, st));
    }
    FinalArgs fin{};
    fin.C = C;
    fin.G = G;
    fin.X = reinterpret_cast<const float *>(ws + lo.X);
    fin.sc = sc;
    fin.gd = dpd->g;
    fin.cams = dpd->cam;
    return run_denoise(ctx, reinterpret_cast<const float *>(ws + lo.X), H, W, P, prm, win, sc, 1, ws, lo, fin, true,
                       st, nullptr, nullptr, fused ? kDenoiseAfterL1Analysis : kDenoiseAll);
}

prnu_status check_camera(const prnu_camera &c, const prnu_params *params) {
    prnu_status s;
    if ((s = check_geometry(c.H, c.W, c.C)) != PRNU_OK) return s;
    if ((s = check_params(params, c.H, c.W, nullptr)) != PRNU_OK) return s;
    if (!c.num || !c.den) return fail(PRNU_EINVAL, "camera num/den is NULL");
    const int fes = params->frame_dtype == PRNU_FRAMES_F16 ? 2 : 1;
    return check_frames(c.frames, c.m, c.H, c.W, c.C, c.frame_stride, c.row_pitch, c.d, fes);
}

size_t multi_layout_bytes(int H, int W, int C, const prnu_params *p, int groups) {
    return align_up(make_layout(H, W, (long long)groups * C, p->levels, true, p->dtype).end, kAlign) +
           sizeof(PassDesc);
}

}  // namespace

// Debug-word readers of the translation units (debug.cuh).
namespace prnu {
std::vector<std::pair<const char *, DebugReader>> &debug_registry() {
    static std::vector<std::pair<const char *, DebugReader>> r;
    return r;
}
void debug_register(const char *unit, DebugReader fn) { debug_registry().emplace_back(unit, fn); }
}  // namespace prnu

// Accessors for the allocation-free entry point (prnu_static.cu).
namespace prnu {
int ctx_device(const prnu_ctx *ctx) { return ctx->device; }
void **ctx_static_scratch(prnu_ctx *ctx) { return &ctx->static_scratch; }
// Validates a residual request the way prnu_denoise_residual does (NULL
// pointers, aliasing, geometry, parameters), so that nothing is resolved or
// launched for invalid input, and returns the bytes of intermediates it
// needs with the requested subband storage type.
prnu_status check_residual_request(const float *img, int H, int W, int C, const prnu_params *params,
                                   const float *residual_out, size_t *need) {
    if (!img || !residual_out) return fail(PRNU_EINVAL, "img/residual_out is NULL");
    if ((const void *)img == (const void *)residual_out) return fail(PRNU_EINVAL, "img and residual_out alias");
    prnu_status s;
    if ((s = check_geometry(H, W, C)) != PRNU_OK) return s;
    if ((s = check_params(params, H, W, nullptr)) != PRNU_OK) return s;
    *need = make_layout(H, W, C, params->levels, false, params->dtype).end;
    return PRNU_OK;
}
prnu_status set_last_error(prnu_status s, const char *msg) { return fail(s, "%s", msg); }
}  // namespace prnu

// ===========================================================================
extern "C" {

prnu_status prnu_default_params(prnu_params *p) {
    if (!p) return fail(PRNU_EINVAL, "params is NULL");
    p->levels = 4;
    p->sigma0 = 3.0f;
    p->n_windows = 4;
    p->windows[0] = 3;
    p->windows[1] = 5;
    p->windows[2] = 7;
    p->windows[3] = 9;
    p->pad_mode = 0;
    p->dtype = PRNU_DTYPE_F32;
    p->frame_dtype = PRNU_FRAMES_U8;
    p->compensated = 0;
    p->sda_blocks_per_sm = 0;
    p->pipeline_passes = 0;
    p->sda_fusion = 0;
    return PRNU_OK;
}

prnu_status prnu_create(prnu_ctx **out, int device) {
    if (!out) return fail(PRNU_EINVAL, "out is NULL");
    *out = nullptr;
    int n = 0;
    CU(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(PRNU_EINVAL, "device %d out of range (%d devices)", device, n);
    DeviceGuard g(device);
    if (!g.ok) return fail(PRNU_ECUDA, "cudaSetDevice(%d) failed", device);
    prnu_ctx *c = new prnu_ctx;
    c->device = device;
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete c;
        return fail(PRNU_ECUDA, "cannot query SM count");
    }
    if (!derive_filter(c->h64)) {
        delete c;
        return fail(PRNU_ECUDA, "filter bank derivation did not converge");
    }
    for (int k = 0; k < kTaps; ++k) {
        c->filt.h[k] = (float)c->h64[k];
        c->filt.g[k] = (float)((k % 2 ? -1.0 : 1.0) * c->h64[kTaps - 1 - k]);
        c->filt.hg[k][0] = c->filt.h[k];
        c->filt.hg[k][1] = c->filt.g[k];
    }
    if (cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return fail(PRNU_ECUDA, "cannot create copy stream");
    }
    for (int i = 0; i < 2; ++i) {
        cudaEventCreateWithFlags(&c->ev_copied[i], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&c->ev_free[i], cudaEventDisableTiming);
    }
    *out = c;
    return PRNU_OK;
}

void prnu_destroy(prnu_ctx *ctx) {
    if (!ctx) return;
    {
        DeviceGuard g(ctx->device);
        for (auto &kv : ctx->plans) cufftDestroy(kv.second);
        if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
        for (int i = 0; i < 2; ++i) {
            if (ctx->ev_copied[i]) cudaEventDestroy(ctx->ev_copied[i]);
            if (ctx->ev_free[i]) cudaEventDestroy(ctx->ev_free[i]);
        }
        for (auto &r : ctx->recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (auto e : ctx->pool) cudaEventDestroy(e);
    }
    delete ctx;
}

const char *prnu_last_error(const prnu_ctx *) { return tl_err.c_str(); }

prnu_status prnu_workspace_size(prnu_ctx *ctx, int H, int W, int C, const prnu_params *params, int images_per_pass,
                                size_t *bytes) {
    if (!ctx || !bytes) return fail(PRNU_EINVAL, "ctx/bytes is NULL");
    prnu_status s;
    if ((s = check_geometry(H, W, C)) != PRNU_OK) return s;
    if ((s = check_params(params, H, W, nullptr)) != PRNU_OK) return s;
    if (images_per_pass < 1) return fail(PRNU_EINVAL, "images_per_pass must be >= 1");
    DeviceGuard g(ctx->device);
    size_t need = make_layout(H, W, (long long)images_per_pass * C, params->levels, true, params->dtype).end;
    FftLayout f;
    if ((s = fft_layout(ctx, H, W, images_per_pass, &f)) != PRNU_OK) return s;
    need = std::max(need, f.end);
    *bytes = need;
    return PRNU_OK;
}

prnu_status prnu_workspace_size_host(prnu_ctx *ctx, int H, int W, int C, int d, const prnu_params *params,
                                     int groups_per_pass, size_t *bytes) {
    if (!ctx || !bytes) return fail(PRNU_EINVAL, "ctx/bytes is NULL");
    prnu_status s;
    if ((s = check_geometry(H, W, C)) != PRNU_OK) return s;
    if ((s = check_params(params, H, W, nullptr)) != PRNU_OK) return s;
    if (groups_per_pass < 1 || d < 1) return fail(PRNU_EINVAL, "groups_per_pass and d must be >= 1");
    const size_t frame = (size_t)H * W * C;
    const size_t stage = align_up((size_t)groups_per_pass * d * frame, kAlign);
    *bytes = 2 * stage + make_layout(H, W, (long long)groups_per_pass * C, params->levels, true, params->dtype).end;
    return PRNU_OK;
}

prnu_status prnu_sda_average(prnu_ctx *ctx, const uint8_t *frames, int m, int H, int W, int C, size_t frame_stride,
                             size_t row_pitch, int d, float *sda_out, void *stream) {
    if (!ctx || !sda_out) return fail(PRNU_EINVAL, "ctx/sda_out is NULL");
    prnu_status s;
    if ((s = check_geometry(H, W, C)) != PRNU_OK) return s;
    if ((s = check_frames(frames, m, H, W, C, frame_stride, row_pitch, d)) != PRNU_OK) return s;
    DeviceGuard g(ctx->device);
    SdaArgs a{};
    a.frames = frames;
    a.frame_stride = (long long)frame_stride;
    a.row_pitch = (long long)row_pitch;
    a.m = m;
    a.H = H;
    a.W = W;
    a.C = C;
    a.d = d;
    a.g0 = 0;
    a.G = (m + d - 1) / d;
    a.out = sda_out;
    a.mean = 1;
    a.frame_half = 0;
    Launch t(ctx, "sda_mean", S(stream), 1, (double)m * H * W * C + (double)a.G * C * H * W * 4);
    CU(launch_sda(a, ctx->sms, S(stream)));
    return PRNU_OK;
}

prnu_status prnu_denoise_residual_batch(prnu_ctx *ctx, const float *img, int n, int H, int W, int C,
                                        const prnu_params *params, float *residual_out, void *ws, size_t ws_bytes,
                                        void *stream) {
    if (!ctx || !img || !residual_out) return fail(PRNU_EINVAL, "ctx/img/residual_out is NULL");
    if ((const void *)img == (const void *)residual_out) return fail(PRNU_EINVAL, "img and residual_out alias");
    if (n < 1) return fail(PRNU_EINVAL, "n must be >= 1");
    prnu_status s;
    Win win;
    if ((s = check_geometry(H, W, C)) != PRNU_OK) return s;
    if ((s = check_params(params, H, W, &win)) != PRNU_OK) return s;
    const Layout lo = make_layout(H, W, (long long)n * C, params->levels, false, params->dtype);
    if ((s = check_ws(ws, ws_bytes, lo.end)) != PRNU_OK) return s;
    DeviceGuard g(ctx->device);
    FinalArgs fin{};
    fin.C = C;
    fin.G = n;
    fin.res_out = residual_out;
    fin.sc = PlaneScale{1, 1, 0, C, nullptr};
    return run_denoise(ctx, img, H, W, n * C, *params, win, fin.sc, 0, static_cast<char *>(ws), lo, fin, false,
                       S(stream));
}

prnu_status prnu_denoise_residual(prnu_ctx *ctx, const float *img, int H, int W, int C, const prnu_params *params,
                                  float *residual_out, void *ws, size_t ws_bytes, void *stream) {
    return prnu_denoise_residual_batch(ctx, img, 1, H, W, C, params, residual_out, ws, ws_bytes, stream);
}

prnu_status prnu_fingerprint_accumulate(prnu_ctx *ctx, const uint8_t *frames, int m, int H, int W, int C,
                                        size_t frame_stride, size_t row_pitch, int d, const prnu_params *params,
                                        float *num, float *den, void *ws, size_t ws_bytes, void *stream) {
    if (!ctx || !num || !den) return fail(PRNU_EINVAL, "ctx/num/den is NULL");
    prnu_status s;
    Win win;
    if ((s = check_geometry(H, W, C)) != PRNU_OK) return s;
    if ((s = check_params(params, H, W, &win)) != PRNU_OK) return s;
    const int fes = params->frame_dtype == PRNU_FRAMES_F16 ? 2 : 1;
    if ((s = check_frames(frames, m, H, W, C, frame_stride, row_pitch, d, fes)) != PRNU_OK) return s;
    const int g = (m + d - 1) / d;
    const int Gp = groups_fitting(H, W, C, params->levels, ws_bytes, g, params->dtype);
    if (Gp < 1) return check_ws(ws, ws_bytes, make_layout(H, W, C, params->levels, true, params->dtype).end);
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(PRNU_EINVAL, "workspace must be 256-byte aligned");
    DeviceGuard gd(ctx->device);
    if (params->pipeline_passes >= 2 && g >= 2) {
        // two pass layouts: the sums of pass k+1 on the side stream beside the denoising of pass k
        const int want = (g + params->pipeline_passes - 1) / params->pipeline_passes;
        const int Gp2 = groups_fitting(H, W, C, params->levels, ws_bytes / 2 / kAlign * kAlign, want, params->dtype);
        if (Gp2 >= 1)
            return accumulate_pipelined(ctx, frames, m, H, W, C, frame_stride, row_pitch, d, g, Gp2, *params, win, num,
                                        den, static_cast<char *>(ws),
                                        params->sda_blocks_per_sm > 0 ? params->sda_blocks_per_sm : kPipeSdaBlocks,
                                        S(stream));
    }
    for (int g0 = 0; g0 < g; g0 += Gp) {
        const int G = std::min(Gp, g - g0);
        if ((s = accumulate_pass(ctx, frames, m, H, W, C, frame_stride, row_pitch, d, g0, G, *params, win, num, den,
                                 static_cast<char *>(ws), S(stream))) != PRNU_OK)
            return s;
    }
    return PRNU_OK;
}

prnu_status prnu_fingerprint_accumulate_host(prnu_ctx *ctx, const uint8_t *host_frames, int m, int H, int W, int C,
                                             size_t frame_stride, size_t row_pitch, int d, const prnu_params *params,
                                             float *num, float *den, void *ws, size_t ws_bytes, void *stream) {
    if (!ctx || !num || !den) return fail(PRNU_EINVAL, "ctx/num/den is NULL");
    prnu_status s;
    Win win;
    if ((s = check_geometry(H, W, C)) != PRNU_OK) return s;
    if ((s = check_params(params, H, W, &win)) != PRNU_OK) return s;
    const int fes = params->frame_dtype == PRNU_FRAMES_F16 ? 2 : 1;
    if ((s = check_frames(host_frames, m, H, W, C, frame_stride, row_pitch, d, fes)) != PRNU_OK) return s;
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(PRNU_EINVAL, "workspace must be 256-byte aligned");
    const int g = (m + d - 1) / d;
    DeviceGuard gd(ctx->device);
    cudaStream_t st = S(stream);
    {
        // Page-locked host frames are read in place by the kernels (through
        // their device-visible address over the host link): no staging copy,
        // and the whole workspace holds pass layouts.
        cudaPointerAttributes attr{};
        if (cudaPointerGetAttributes(&attr, host_frames) == cudaSuccess && attr.type == cudaMemoryTypeHost &&
            attr.devicePointer) {
            const uint8_t *dev = static_cast<const uint8_t *>(attr.devicePointer);
            // Two pass layouts: the sums of pass k+1 are read over the link (on the
            // context's side stream, two blocks per SM are enough for its bandwidth)
            // while pass k is denoised on `stream`.
            // at least four passes, so that all but the last pass's denoise hides behind the reads
            const int Gp2 = groups_fitting(H, W, C, params->levels, ws_bytes / 2 / kAlign * kAlign,
                                           std::max(1, (g + 3) / 4), params->dtype);
            if (Gp2 >= 1 && g > Gp2)
                return accumulate_pipelined(ctx, dev, m, H, W, C, frame_stride, row_pitch, d, g, Gp2, *params, win,
                                            num, den, static_cast<char *>(ws),
                                            params->sda_blocks_per_sm > 0 ? params->sda_blocks_per_sm : 2, st);
            const int Gp = groups_fitting(H, W, C, params->levels, ws_bytes, g, params->dtype);
            if (Gp < 1) return check_ws(ws, ws_bytes, make_layout(H, W, C, params->levels, true, params->dtype).end);
            for (int g0 = 0; g0 < g; g0 += Gp)
                if ((s = accumulate_pass(ctx, dev, m, H, W, C, frame_stride, row_pitch, d, g0, std::min(Gp, g - g0),
                                         *params, win, num, den, static_cast<char *>(ws), st, false)) != PRNU_OK)
                    return s;
            return PRNU_OK;
        }
        cudaGetLastError();  // pageable memory: clear the query's error state, stage through the device
    }
    const size_t fbytes = (size_t)H * W * C * fes;  // staged frames are packed
    // largest groups-per-pass with two staging buffers and the pass layout
    int Gp = 0;
    for (int lo = 1, hi = g; lo <= hi;) {
        const int mid = (lo + hi) / 2;
        const size_t stage = align_up((size_t)mid * d * fbytes, kAlign);
        const size_t need = 2 * stage + make_layout(H, W, (long long)mid * C, params->levels, true, params->dtype).end;
        if (need <= ws_bytes) {
            Gp = mid;
            lo = mid + 1;
        } else {
            hi = mid - 1;
        }
    }
    if (Gp < 1) {
        const size_t need =
            2 * align_up((size_t)d * fbytes, kAlign) + make_layout(H, W, C, params->levels, true, params->dtype).end;
        return fail(PRNU_ENOSPC, "workspace too small: need %zu bytes, got %zu", need, ws_bytes);
    }
    char *base = static_cast<char *>(ws);
    const size_t stage = align_up((size_t)Gp * d * fbytes, kAlign);
    uint8_t *buf[2] = {reinterpret_cast<uint8_t *>(base), reinterpret_cast<uint8_t *>(base + stage)};
    char *rest = base + 2 * stage;
    const size_t rowb = (size_t)W * C * fes;
    const bool packed = row_pitch == rowb && (m == 1 || frame_stride == (size_t)H * rowb);
    int k = 0;
    for (int g0 = 0; g0 < g; g0 += Gp, ++k) {
        const int G = std::min(Gp, g - g0);
        const int j0 = g0 * d, j1 = std::min(m, (g0 + G) * d);
        const int b = k & 1;
        CU(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_free[b], 0));
        if (packed) {
            CU(cudaMemcpyAsync(buf[b], host_frames + (size_t)j0 * fbytes, (size_t)(j1 - j0) * fbytes,
                               cudaMemcpyHostToDevice, ctx->copy_stream));
        } else {
            for (int j = j0; j < j1; ++j)
                CU(cudaMemcpy2DAsync(buf[b] + (size_t)(j - j0) * fbytes, rowb,
                                     host_frames + (size_t)j * frame_stride, row_pitch, rowb, H,
                                     cudaMemcpyHostToDevice, ctx->copy_stream));
        }
        CU(cudaEventRecord(ctx->ev_copied[b], ctx->copy_stream));
        CU(cudaStreamWaitEvent(st, ctx->ev_copied[b], 0));
        // the staged chunk holds frames j0 .. j1-1, i.e. groups 0..G-1 of a
        // sequence of (j1 - j0) frames
        if ((s = accumulate_pass(ctx, buf[b], j1 - j0, H, W, C, fbytes, rowb, d, 0, G, *params, win, num,
                                 den, rest, st)) != PRNU_OK)
            return s;
        CU(cudaEventRecord(ctx->ev_free[b], st));
    }
    return PRNU_OK;
}

prnu_status prnu_fingerprint_finalize(prnu_ctx *ctx, const float *num, const float *den, int H, int W, int C,
                                      unsigned flags, const prnu_params *params, float *K_out, void *ws,
                                      size_t ws_bytes, void *stream) {
    if (!ctx || !num || !den || !K_out) return fail(PRNU_EINVAL, "ctx/num/den/K_out is NULL");
    prnu_status s;
    Win win;
    if ((s = check_geometry(H, W, C)) != PRNU_OK) return s;
    if (flags & ~(PRNU_ZERO_MEAN | PRNU_WIENER_DFT | PRNU_TO_GRAY)) return fail(PRNU_EINVAL, "unknown flags");
    if ((flags & PRNU_TO_GRAY) && C != 3) return fail(PRNU_EINVAL, "PRNU_TO_GRAY needs C == 3");
    if ((flags & PRNU_WIENER_DFT) && (s = check_params(params, H, W, &win)) != PRNU_OK) return s;
    DeviceGuard g(ctx->device);
    cudaStream_t st = S(stream);
    const long long hw = (long long)H * W;
    const int Cout = (flags & PRNU_TO_GRAY) ? 1 : C;
    FftLayout f{};
    if (flags & (PRNU_ZERO_MEAN | PRNU_WIENER_DFT)) {
        if ((s = fft_layout(ctx, H, W, 1, &f)) != PRNU_OK) return s;
        if ((s = check_ws(ws, ws_bytes, f.end)) != PRNU_OK) return s;
    }
    char *b = static_cast<char *>(ws);
    {
        Launch t(ctx, "finalize_divide", st, 1, (double)hw * 4 * (2 * C + Cout));
        const bool comp = params && params->compensated;
        CU(launch_divide(num, den, comp ? num + C * hw : nullptr, comp ? den + C * hw : nullptr, hw, C,
                         (flags & PRNU_TO_GRAY) ? 1 : 0, K_out, ctx->sms, st));
    }
    for (int c = 0; c < Cout; ++c) {
        float *K = K_out + c * hw;
        if (flags & PRNU_ZERO_MEAN)
            {
                Launch t(ctx, "finalize_zero_mean", st, 4, (double)hw * 4 * 4);
                CU(launch_zero_mean(K, H, W, reinterpret_cast<double *>(b + f.colmean),
                                    reinterpret_cast<double *>(b + f.rowmean),
                                    reinterpret_cast<double *>(b + f.colpart), ctx->sms, st));
            }
        if (flags & PRNU_WIENER_DFT) {
            cufftHandle r2c, c2r;
            size_t work;
            if ((s = get_plan(ctx, H, W, CUFFT_R2C, 1, &r2c, &work)) != PRNU_OK) return s;
            if ((s = get_plan(ctx, H, W, CUFFT_C2R, 1, &c2r, &work)) != PRNU_OK) return s;
            cufftComplex *F = reinterpret_cast<cufftComplex *>(b + f.cplx);  // half spectrum
            float *M = reinterpret_cast<float *>(b + f.real);
            float *Mn = M + hw;
            double *mom = reinterpret_cast<double *>(b + f.mom0);
            {
                const bool centred = (flags & PRNU_ZERO_MEAN) != 0;  // K's mean was just removed
                Launch t(ctx, "mean_var", st, centred ? 2 : 4);
                CU(launch_mean_var(K, hw, reinterpret_cast<double *>(b + f.part), kRedBlocks,
                                   reinterpret_cast<double *>(b + f.tmp), mom, st, centred));
            }
            {
                Launch t(ctx, "cufft_r2c", st, 1);
                CUFFT(cufftSetStream(r2c, st));
                CUFFT(cufftSetWorkArea(r2c, b + f.work));
                CUFFT(cufftExecR2C(r2c, K, F));
            }
            {
                Launch t(ctx, "wiener_magnitude", st, 1);
                CU(launch_magnitude_half(F, H, W, (float)(1.0 / std::sqrt((double)hw)), M, ctx->sms, st));
            }
            ShrinkArgs sa{};
            sa.in = M;
            sa.out = Mn;
            sa.R = H;
            sa.Cc = W;
            sa.nplanes = 1;
            sa.s2 = 0.f;
            sa.s2_dev = mom;  // variance of K
            sa.win = win;
            {
                Launch t(ctx, "wiener_shrink", st);
                CU(launch_shrink(sa, st));
            }
            {
                Launch t(ctx, "wiener_ratio", st, 1);  // with the inverse transform's 1/N
                CU(launch_apply_ratio_half(F, M, Mn, H, W, (float)(1.0 / (double)hw), ctx->sms, st));
            }
            {
                Launch t(ctx, "cufft_c2r", st, 1);
                CUFFT(cufftSetStream(c2r, st));
                CUFFT(cufftSetWorkArea(c2r, b + f.work));
                CUFFT(cufftExecC2R(c2r, F, K));
            }
        }
    }
    return PRNU_OK;
}

namespace {
prnu_status pce_correlate_cufft(prnu_ctx *ctx, int n, int H, int W, int nbhd, const FftLayout &f, char *b,
                                const double *part_m, int nbm, cudaStream_t st);
prnu_status pce_to_host(int n, int W, long long hw, int nbhd, const char *scal, double *pce_out, double *ncc_out,
                        int *peak_yx, cudaStream_t st);

// From X, Y in f.real (X_0..X_{n-1}, then Y_0..Y_{n-1}) and the moment
// partials (nbm per query at part_m): cross-correlation, energy, PCE / NCC
// / peak, to the host (synchronising the stream) or, with device_out, to the
// device pointers.
prnu_status pce_finish(prnu_ctx *ctx, int n, int H, int W, int nbhd, const FftLayout &f, char *b,
                       const double *part_m, int nbm, double *pce_out, double *ncc_out, int *peak_yx,
                       cudaStream_t st, bool device_out = false) {
    prnu_status s;
    const long long hw = (long long)H * W;
    const long long nh = (long long)H * (W / 2 + 1);
    const float *X = reinterpret_cast<const float *>(b + f.real);
    if (f.own_fft) {
        // correlation by our own row / column FFTs; the plane is never stored
        float2 *F = reinterpret_cast<float2 *>(b + f.cplx);
        float2 *tw = reinterpret_cast<float2 *>(b + f.tw);
        double *pe = reinterpret_cast<double *>(b + f.pe);
        float *pv = reinterpret_cast<float *>(b + f.pv), *c0 = reinterpret_cast<float *>(b + f.c0);
        long long *pi = reinterpret_cast<long long *>(b + f.pi);
        const int nbr = corr_rows_blocks(H, W, f.nb);
        {
            Launch t(ctx, "pce_fft_rows", st, 2, (double)n * (2.0 * hw * 4 + 2.0 * nh * 8));
            CU(launch_corr_fft(X, F, tw, n, H, W, nbhd / 2, nbr, pe, pv, pi, c0, ctx->sms, st, 0));
        }
        {
            Launch t(ctx, "pce_fft_columns", st, 1, (double)n * 3.0 * nh * 8);
            CU(launch_corr_fft(X, F, tw, n, H, W, nbhd / 2, nbr, pe, pv, pi, c0, ctx->sms, st, 1));
        }
        {
            Launch t(ctx, "pce_fft_rows_inverse", st, 1, (double)n * nh * 8);
            CU(launch_corr_fft(X, F, tw, n, H, W, nbhd / 2, nbr, pe, pv, pi, c0, ctx->sms, st, 2));
        }
        {
            Launch t(ctx, "pce_final", st);
            CU(launch_pce_final(c0, 1, n, pe, pv, pi, nbr, part_m, nbm, b + f.scal, st));
        }
    } else {
        if ((s = pce_correlate_cufft(ctx, n, H, W, nbhd, f, b, part_m, nbm, st)) != PRNU_OK) return s;
    }
    if (device_out) {  // outputs stay on the device: nothing synchronises (graph-capturable)
        Launch t(ctx, "pce_outputs", st);
        CU(launch_pce_outputs(b + f.scal, n, hw, W, nbhd, pce_out, ncc_out, peak_yx, st));
        return PRNU_OK;
    }
    return pce_to_host(n, W, hw, nbhd, b + f.scal, pce_out, ncc_out, peak_yx, st);
}

// cuFFT correlation for geometries the own FFT does not cover
prnu_status pce_correlate_cufft(prnu_ctx *ctx, int n, int H, int W, int nbhd, const FftLayout &f, char *b,
                                const double *part_m, int nbm, cudaStream_t st) {
    prnu_status s;
    const long long hw = (long long)H * W;
    const long long nh = (long long)H * (W / 2 + 1);
    float *X = reinterpret_cast<float *>(b + f.real);
    cufftComplex *FX = reinterpret_cast<cufftComplex *>(b + f.cplx);
    cufftHandle r2c, c2r;
    size_t w1, w2;
    if ((s = get_plan(ctx, H, W, CUFFT_R2C, 2 * n, &r2c, &w1)) != PRNU_OK) return s;
    if ((s = get_plan(ctx, H, W, CUFFT_C2R, n, &c2r, &w2)) != PRNU_OK) return s;
    {
        Launch t(ctx, "cufft_r2c", st);
        CUFFT(cufftSetStream(r2c, st));
        CUFFT(cufftSetWorkArea(r2c, b + f.work));
        CUFFT(cufftExecR2C(r2c, X, FX));  // 2n half spectra: FX_i, then FY_i
    }
    {
        Launch t(ctx, "pce_cross_spectrum", st, 1, (double)n * nh * 24);
        CU(launch_cross_spectrum(FX, FX + n * nh, nh, n, FX, ctx->sms, st));
    }
    {
        Launch t(ctx, "cufft_c2r", st);
        CUFFT(cufftSetStream(c2r, st));
        CUFFT(cufftSetWorkArea(c2r, b + f.work));
        CUFFT(cufftExecC2R(c2r, FX, X));  // X_i now holds hw * C_i(s)
    }
    {
        Launch t(ctx, "pce_reduce", st, 2, (double)n * hw * 4);
        CU(launch_pce_reduce(X, H, W, nbhd / 2, n, f.nb, reinterpret_cast<double *>(b + f.pe),
                             reinterpret_cast<float *>(b + f.pv), reinterpret_cast<long long *>(b + f.pi), part_m,
                             nbm, b + f.scal, st));
    }
    return PRNU_OK;
}

// PCE / NCC / peak of the n queries to the host (synchronises the stream)
prnu_status pce_to_host(int n, int W, long long hw, int nbhd, const char *scal, double *pce_out, double *ncc_out,
                        int *peak_yx, cudaStream_t st) {
    std::vector<unsigned char> host((size_t)n * pce_scalars_bytes());
    CU(cudaMemcpyAsync(host.data(), scal, host.size(), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    const double N = (double)hw;
    const double outside = N - (double)nbhd * nbhd;
    for (int q = 0; q < n; ++q) {
        double c0, energy, sx, sxx, sy, syy;
        long long pidx;
        pce_unpack(host.data(), q, &c0, &energy, &pidx, &sx, &sxx, &sy, &syy);
        // c0 and energy carry the unnormalised inverse-FFT factor N (c0) and
        // N^2 (energy): PCE is invariant to it, NCC divides it out.
        pce_out[q] = energy > 0.0 ? (c0 >= 0 ? 1.0 : -1.0) * c0 * c0 * outside / energy : 0.0;
        if (ncc_out) {
            const double nx2 = sxx - sx * sx / N, ny2 = syy - sy * sy / N;
            ncc_out[q] = (nx2 > 0.0 && ny2 > 0.0) ? (c0 / N) / std::sqrt(nx2 * ny2) : 0.0;
        }
        if (peak_yx) {
            peak_yx[2 * q] = (int)(pidx / W);
            peak_yx[2 * q + 1] = (int)(pidx % W);
        }
    }
    return PRNU_OK;
}

prnu_status pce_impl(prnu_ctx *ctx, const float *K, long long k_stride, const float *residual_q, const float *img_q,
                     int n, int H, int W, int C, int nbhd, double *pce_out, double *ncc_out, int *peak_yx, void *ws,
                     size_t ws_bytes, void *stream) {
    if (!ctx || !K || !residual_q || !img_q || !pce_out) return fail(PRNU_EINVAL, "NULL argument");
    if (n < 1) return fail(PRNU_EINVAL, "n must be >= 1");
    prnu_status s;
    if ((s = check_geometry(H, W, C)) != PRNU_OK) return s;
    if (nbhd < 1 || nbhd % 2 == 0 || nbhd > H || nbhd > W) return fail(PRNU_EINVAL, "nbhd must be odd and <= min(H, W)");
    DeviceGuard g(ctx->device);
    FftLayout f;
    if ((s = fft_layout(ctx, H, W, n, &f)) != PRNU_OK) return s;
    if ((s = check_ws(ws, ws_bytes, f.end)) != PRNU_OK) return s;
    cudaStream_t st = S(stream);
    char *b = static_cast<char *>(ws);
    const long long hw = (long long)H * W;
    float *X = reinterpret_cast<float *>(b + f.real);  // X_0..X_{n-1}, then Y_0..Y_{n-1}
    float *Y = X + n * hw;
    {
        Launch t(ctx, "pce_prep", st, 1, (double)n * hw * 4 * (2 * C + 2) + (double)hw * 4);
        CU(launch_pce_prep(K, k_stride, residual_q, img_q, hw, C, n, f.nbm, X, Y,
                           reinterpret_cast<double *>(b + f.pm), st));
    }
    return pce_finish(ctx, n, H, W, nbhd, f, b, reinterpret_cast<double *>(b + f.pm), f.nbm, pce_out, ncc_out,
                      peak_yx, st);
}

// Workspace of prnu_pce_match_images: the denoise layout of n*C planes, then
// the FFT layout of n queries, then the moment partials of the fused kernel.
struct PceImagesLayout {
    Layout den;
    FftLayout fft;
    size_t fft_off = 0, pm = 0, end = 0;
    int nbm = 0;
};

prnu_status pce_images_layout(prnu_ctx *ctx, int H, int W, int C, const prnu_params *params, int n,
                              PceImagesLayout *out) {
    PceImagesLayout p;
    prnu_status s;
    p.den = make_layout(H, W, (long long)n * C, params->levels, false, PRNU_DTYPE_F32);
    p.fft_off = align_up(p.den.end, kAlign);
    if ((s = fft_layout(ctx, H, W, n, &p.fft)) != PRNU_OK) return s;
    const int L = params->levels;
    p.nbm = final_pce_blocks(padded(H, L) / 2, padded(W, L) / 2);
    p.pm = align_up(p.fft_off + p.fft.end, kAlign);
    p.end = p.pm + (size_t)n * p.nbm * 4 * sizeof(double);
    *out = p;
    return PRNU_OK;
}

}  // namespace

prnu_status prnu_workspace_size_pce_images(prnu_ctx *ctx, int H, int W, int C, const prnu_params *params, int n,
                                           size_t *bytes) {
    if (!ctx || !bytes) return fail(PRNU_EINVAL, "NULL argument");
    if (n < 1) return fail(PRNU_EINVAL, "n must be >= 1");
    prnu_status s;
    if ((s = check_geometry(H, W, C)) != PRNU_OK) return s;
    if ((s = check_params(params, H, W, nullptr)) != PRNU_OK) return s;
    DeviceGuard g(ctx->device);
    PceImagesLayout p;
    if ((s = pce_images_layout(ctx, H, W, C, params, n, &p)) != PRNU_OK) return s;
    *bytes = p.end;
    return PRNU_OK;
}

namespace {
prnu_status pce_images_impl(prnu_ctx *ctx, const float *K, const float *img_q, int n, int H, int W, int C,
                            const prnu_params *params, int nbhd, double *pce_out, double *ncc_out, int *peak_yx,
                            void *ws, size_t ws_bytes, void *stream, bool device_out, int phase = kDenoiseAll) {
    if (!ctx || !img_q || (phase != kDenoiseUpToLevel2 && (!K || !pce_out))) return fail(PRNU_EINVAL, "NULL argument");
    if (n < 1) return fail(PRNU_EINVAL, "n must be >= 1");
    prnu_status s;
    Win win;
    if ((s = check_geometry(H, W, C)) != PRNU_OK) return s;
    if ((s = check_params(params, H, W, &win)) != PRNU_OK) return s;
    if (params->dtype != PRNU_DTYPE_F32)
        return fail(PRNU_EUNSUPPORTED, "prnu_pce_match_images needs float32 subbands (use prnu_denoise_residual_batch "
                                       "and prnu_pce_match_batch)");
    if (nbhd < 1 || nbhd % 2 == 0 || nbhd > H || nbhd > W) return fail(PRNU_EINVAL, "nbhd must be odd and <= min(H, W)");
    DeviceGuard g(ctx->device);
    PceImagesLayout p;
    if ((s = pce_images_layout(ctx, H, W, C, params, n, &p)) != PRNU_OK) return s;
    if ((s = check_ws(ws, ws_bytes, p.end)) != PRNU_OK) return s;
    cudaStream_t st = S(stream);
    char *b = static_cast<char *>(ws);
    const long long hw = (long long)H * W;
    float *X = reinterpret_cast<float *>(b + p.fft_off + p.fft.real);
    FinalArgs fin{};
    fin.C = C;
    fin.G = n;
    fin.sc = PlaneScale{1, 1, 0, C, nullptr};
    fin.pce = 1;
    fin.Kq = K;
    fin.k_stride = 0;
    fin.Iq = img_q;
    fin.Xo = X;
    fin.Yo = X + n * hw;
    fin.part_m = reinterpret_cast<double *>(b + p.pm);
    if ((s = run_denoise(ctx, img_q, H, W, n * C, *params, win, fin.sc, 0, b, p.den, fin, false, st, nullptr,
                         nullptr, phase)) != PRNU_OK)
        return s;
    if (phase == kDenoiseUpToLevel2) return PRNU_OK;
    return pce_finish(ctx, n, H, W, nbhd, p.fft, b + p.fft_off, fin.part_m, p.nbm, pce_out, ncc_out, peak_yx, st,
                      device_out);
}
}  // namespace

prnu_status prnu_pce_images_prepare(prnu_ctx *ctx, const float *img_q, int n, int H, int W, int C,
                                    const prnu_params *params, void *ws, size_t ws_bytes, void *stream) {
    return pce_images_impl(ctx, nullptr, img_q, n, H, W, C, params, 1, nullptr, nullptr, nullptr, ws, ws_bytes,
                           stream, true, kDenoiseUpToLevel2);
}

prnu_status prnu_pce_images_finish_async(prnu_ctx *ctx, const float *K, const float *img_q, int n, int H, int W,
                                         int C, const prnu_params *params, int nbhd, double *pce_dev,
                                         double *ncc_dev, int *peak_dev, void *ws, size_t ws_bytes, void *stream) {
    return pce_images_impl(ctx, K, img_q, n, H, W, C, params, nbhd, pce_dev, ncc_dev, peak_dev, ws, ws_bytes, stream,
                           true, kDenoiseLevel1);
}

prnu_status prnu_pce_match_images(prnu_ctx *ctx, const float *K, const float *img_q, int n, int H, int W, int C,
                                  const prnu_params *params, int nbhd, double *pce_out, double *ncc_out,
                                  int *peak_yx, void *ws, size_t ws_bytes, void *stream) {
    return pce_images_impl(ctx, K, img_q, n, H, W, C, params, nbhd, pce_out, ncc_out, peak_yx, ws, ws_bytes, stream,
                           false);
}

prnu_status prnu_pce_match_images_async(prnu_ctx *ctx, const float *K, const float *img_q, int n, int H, int W,
                                        int C, const prnu_params *params, int nbhd, double *pce_dev, double *ncc_dev,
                                        int *peak_dev, void *ws, size_t ws_bytes, void *stream) {
    return pce_images_impl(ctx, K, img_q, n, H, W, C, params, nbhd, pce_dev, ncc_dev, peak_dev, ws, ws_bytes, stream,
                           true);
}

prnu_status prnu_pce_match_batch(prnu_ctx *ctx, const float *K, const float *residual_q, const float *img_q, int n,
                                 int H, int W, int C, int nbhd, double *pce_out, double *ncc_out, int *peak_yx,
                                 void *ws, size_t ws_bytes, void *stream) {
    return pce_impl(ctx, K, 0, residual_q, img_q, n, H, W, C, nbhd, pce_out, ncc_out, peak_yx, ws, ws_bytes, stream);
}

prnu_status prnu_pce_match_pairs(prnu_ctx *ctx, const float *K, const float *residual_q, const float *img_q, int n,
                                 int H, int W, int C, int nbhd, double *pce_out, double *ncc_out, int *peak_yx,
                                 void *ws, size_t ws_bytes, void *stream) {
    return pce_impl(ctx, K, (long long)H * W, residual_q, img_q, n, H, W, C, nbhd, pce_out, ncc_out, peak_yx, ws,
                    ws_bytes, stream);
}

prnu_status prnu_pce_match(prnu_ctx *ctx, const float *K, const float *residual_q, const float *img_q, int H, int W,
                           int C, int nbhd, double *pce_out, double *ncc_out, int *peak_yx, void *ws,
                           size_t ws_bytes, void *stream) {
    return prnu_pce_match_batch(ctx, K, residual_q, img_q, 1, H, W, C, nbhd, pce_out, ncc_out, peak_yx, ws,
                                ws_bytes, stream);
}

prnu_status prnu_workspace_size_multi(prnu_ctx *ctx, const prnu_camera *cams, int ncams, const prnu_params *params,
                                      int groups_per_pass, size_t *bytes) {
    if (!ctx || !cams || !bytes || ncams < 1) return fail(PRNU_EINVAL, "NULL argument or ncams < 1");
    if (groups_per_pass < 1 || groups_per_pass > kMaxPassGroups)
        return fail(PRNU_EINVAL, "groups_per_pass must be in [1, %d]", kMaxPassGroups);
    size_t need = 0;
    for (int i = 0; i < ncams; ++i) {
        prnu_status s = check_camera(cams[i], params);
        if (s != PRNU_OK) return s;
        need = std::max(need, multi_layout_bytes(cams[i].H, cams[i].W, cams[i].C, params, groups_per_pass));
    }
    *bytes = need;
    return PRNU_OK;
}

prnu_status prnu_fingerprint_accumulate_multi(prnu_ctx *ctx, const prnu_camera *cams, int ncams,
                                              const prnu_params *params, void *ws, size_t ws_bytes, void *stream) {
    if (!ctx || !cams || ncams < 1) return fail(PRNU_EINVAL, "NULL argument or ncams < 1");
    prnu_status s;
    Win win;
    for (int i = 0; i < ncams; ++i)
        if ((s = check_camera(cams[i], params)) != PRNU_OK) return s;
    if ((s = check_params(params, cams[0].H, cams[0].W, &win)) != PRNU_OK) return s;
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(PRNU_EINVAL, "workspace must be 256-byte aligned");
    DeviceGuard gd(ctx->device);
    cudaStream_t st = S(stream);
    // geometry classes in order of first appearance
    std::vector<int> done(ncams, 0);
    for (int i0 = 0; i0 < ncams; ++i0) {
        if (done[i0]) continue;
        const int H = cams[i0].H, W = cams[i0].W, C = cams[i0].C;
        std::vector<int> members;
        for (int i = i0; i < ncams; ++i)
            if (!done[i] && cams[i].H == H && cams[i].W == W && cams[i].C == C) {
                members.push_back(i);
                done[i] = 1;
            }
        // largest pass that fits the workspace and the descriptor table
        int Gp = 0;
        for (int g = kMaxPassGroups; g >= 1; g = g > 8 ? g * 3 / 4 : g - 1)
            if (multi_layout_bytes(H, W, C, params, g) <= ws_bytes) {
                Gp = g;
                break;
            }
        if (Gp < 1) {
            return fail(PRNU_ENOSPC, "workspace too small: need %zu bytes, got %zu",
                        multi_layout_bytes(H, W, C, params, 1), ws_bytes);
        }
        // walk the groups of the class's cameras, in camera order
        PassDesc pd;
        pd.G = 0;
        pd.ncam = 0;
        auto flush = [&]() -> prnu_status {
            if (pd.G == 0) return PRNU_OK;
            prnu_status r = accumulate_pass_multi(ctx, pd, H, W, C, *params, win, static_cast<char *>(ws), st);
            pd.G = 0;
            pd.ncam = 0;
            return r;
        };
        for (int ci : members) {
            const prnu_camera &c = cams[ci];
            const int g = (c.m + c.d - 1) / c.d;
            for (int k = 0; k < g; ++k) {
                if (pd.G == Gp || (pd.ncam == kMaxPassCams && (pd.ncam == 0 || pd.cam[pd.ncam - 1].num != c.num))) {
                    if ((s = flush()) != PRNU_OK) return s;
                }
                if (pd.ncam == 0 || pd.cam[pd.ncam - 1].num != c.num) {
                    pd.cam[pd.ncam].num = c.num;
                    pd.cam[pd.ncam].den = c.den;
                    ++pd.ncam;
                }
                GroupDesc &gdesc = pd.g[pd.G++];
                const int j0 = k * c.d, j1 = std::min(c.m, j0 + c.d);
                gdesc.frames = c.frames + (size_t)j0 * c.frame_stride;
                gdesc.frame_stride = (long long)c.frame_stride;
                gdesc.row_pitch = (long long)c.row_pitch;
                gdesc.n = j1 - j0;
                gdesc.cam = pd.ncam - 1;
            }
        }
        if ((s = flush()) != PRNU_OK) return s;
    }
    return PRNU_OK;
}

prnu_status prnu_autotune(prnu_ctx *ctx, int H, int W, int C, const prnu_params *params, int images, void *ws,
                          size_t ws_bytes, void *stream, int *shape_out, float *ms_out) {
    if (!ctx) return fail(PRNU_EINVAL, "ctx is NULL");
    prnu_status s;
    if ((s = check_geometry(H, W, C)) != PRNU_OK) return s;
    if ((s = check_params(params, H, W, nullptr)) != PRNU_OK) return s;
    if (images < 1) return fail(PRNU_EINVAL, "images must be >= 1");
    const int P = images * C;
    const Layout lo = make_layout(H, W, P, params->levels, true, params->dtype);
    if ((s = check_ws(ws, ws_bytes, lo.end)) != PRNU_OK) return s;
    DeviceGuard g(ctx->device);
    cudaStream_t st = S(stream);
    char *b = static_cast<char *>(ws);
    const int L = params->levels, Hp = padded(H, L), Wp = padded(W, L);
    const long long A = (long long)(Hp >> 1) * (Wp >> 1);
    const size_t es = subband_bytes(params->dtype);
    CU(cudaMemsetAsync(b + lo.X, 0, (size_t)P * H * W * sizeof(float), st));
    AnaArgs a{};
    a.inh = reinterpret_cast<const float *>(b + lo.X);
    a.R = Hp;
    a.Cc = Wp;
    a.H = H;
    a.W = W;
    a.P = P;
    a.LLh = L > 1 ? reinterpret_cast<float *>(b + lo.LLh[1]) : nullptr;
    a.LLl = L > 1 ? reinterpret_cast<float *>(b + lo.LLl[1]) : nullptr;
    a.LH = b + lo.D[1];
    a.HL = b + lo.D[1] + (size_t)P * A * es;
    a.HH = b + lo.D[1] + 2 * (size_t)P * A * es;
    a.sdt = params->dtype;
    a.sc = PlaneScale{1, 1, 0, C, nullptr};
    a.scale_on = 0;
    a.f = ctx->filt;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    int best = kStreamShapeDefault;
    float best_ms = 1e30f;
    for (int shape = 0; shape < kStreamShapes; ++shape) {
        CU(launch_analysis(a, true, st, shape));  // warm
        CU(cudaEventRecord(e0, st));
        for (int r = 0; r < 3; ++r) CU(launch_analysis(a, true, st, shape));
        CU(cudaEventRecord(e1, st));
        CU(cudaEventSynchronize(e1));
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, e0, e1));
        ms /= 3.f;
        if (ms < best_ms) {
            best_ms = ms;
            best = shape;
        }
    }
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->tuned[std::make_tuple(Hp, Wp, (int)params->dtype)] = best;
    }
    // the other launches, level by level on the pyramid of the zero planes:
    // analysis of levels 2..L, shrink of levels 1..L, synthesis of levels L..2
    CU(launch_analysis(a, true, st, best));  // LL_1 and the level-1 details
    auto time_it = [&](auto &&launch, float *ms) -> prnu_status {
        CU(launch());  // warm
        CU(cudaEventRecord(e0, st));
        for (int r = 0; r < 3; ++r) CU(launch());
        CU(cudaEventRecord(e1, st));
        CU(cudaEventSynchronize(e1));
        CU(cudaEventElapsedTime(ms, e0, e1));
        return PRNU_OK;
    };
    const int sdt = params->dtype;
    auto keep = [&](int kind, int l, int c) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->tuned_lv[std::make_tuple(Hp, Wp, sdt, kind, l)] = c;
    };
    Win win;
    if ((s = check_params(params, H, W, &win)) != PRNU_OK) return s;
    for (int l = 1; l <= L; ++l) {
        const long long Al = (long long)(Hp >> l) * (Wp >> l);
        if (l >= 2) {
            AnaArgs al = a;
            al.inh = reinterpret_cast<const float *>(b + lo.LLh[l - 1]);
            al.inl = reinterpret_cast<const float *>(b + lo.LLl[l - 1]);
            al.R = Hp >> (l - 1);
            al.Cc = Wp >> (l - 1);
            al.LLh = l < L ? reinterpret_cast<float *>(b + lo.LLh[l]) : nullptr;
            al.LLl = l < L ? reinterpret_cast<float *>(b + lo.LLl[l]) : nullptr;
            al.LH = b + lo.D[l];
            al.HL = b + lo.D[l] + (size_t)P * Al * es;
            al.HH = b + lo.D[l] + 2 * (size_t)P * Al * es;
            int bc = 0;
            float bm = 1e30f;
            for (int c = 0; c < kAnaChoices; ++c) {
                float ms = 0.f;
                if ((s = time_it([&] { return launch_analysis(al, false, st, c); }, &ms)) != PRNU_OK) return s;
                if (ms < bm) {
                    bm = ms;
                    bc = c;
                }
            }
            keep(kTuneAnalysis, l, bc);
            CU(launch_analysis(al, false, st, bc));  // this level's outputs for the next one
        }
        ShrinkArgs sa{};
        sa.in = b + lo.D[l];
        sa.out = b + lo.N[l];
        sa.sdt = sdt;
        sa.R = Hp >> l;
        sa.Cc = Wp >> l;
        sa.nplanes = 3 * P;
        sa.s2 = params->sigma0 * params->sigma0;
        sa.win = win;
        int bc = 0;
        float bm = 1e30f;
        for (int c = 0; c < kShrinkChoices; ++c) {
            float ms = 0.f;
            if ((s = time_it([&] { return launch_shrink(sa, st, c); }, &ms)) != PRNU_OK) return s;
            if (ms < bm) {
                bm = ms;
                bc = c;
            }
        }
        keep(kTuneShrink, l, bc);
    }
    for (int l = L; l >= 2; --l) {
        const long long Al = (long long)(Hp >> l) * (Wp >> l);
        SynArgs y{};
        y.LL = l == L ? nullptr : b + lo.Rn[l];
        y.LH = b + lo.N[l];
        y.HL = b + lo.N[l] + (size_t)P * Al * es;
        y.HH = b + lo.N[l] + 2 * (size_t)P * Al * es;
        y.sdt = sdt;
        y.Rc = Hp >> l;
        y.Cc = Wp >> l;
        y.P = P;
        y.out = b + lo.Rn[l - 1];
        y.f = ctx->filt;
        int bc = 0;
        float bm = 1e30f;
        for (int c = 0; c < kSynChoices; ++c) {
            float ms = 0.f;
            if ((s = time_it([&] { return launch_synthesis(y, st, c); }, &ms)) != PRNU_OK) return s;
            if (ms < bm) {
                bm = ms;
                bc = c;
            }
        }
        keep(kTuneSynthesis, l, bc);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (shape_out) *shape_out = best;
    if (ms_out) *ms_out = best_ms;
    return PRNU_OK;
}

prnu_status prnu_autotune_level(prnu_ctx *ctx, int H, int W, const prnu_params *params, int kind, int level,
                                int choice, int *current) {
    if (!ctx) return fail(PRNU_EINVAL, "ctx is NULL");
    prnu_status s;
    if ((s = check_geometry(H, W, 1)) != PRNU_OK) return s;
    if ((s = check_params(params, H, W, nullptr)) != PRNU_OK) return s;
    const int L = params->levels;
    const int nch = kind == kTuneAnalysis ? kAnaChoices : kind == kTuneShrink ? kShrinkChoices
                  : kind == kTuneSynthesis ? kSynChoices : kind == kTuneFinal ? kFinalChoices : 0;
    if (nch == 0)
        return fail(PRNU_EINVAL, "kind must be 0 (analysis), 1 (shrink), 2 (synthesis) or 3 (level-1 MLE step)");
    const int lmin = kind == kTuneShrink || kind == kTuneFinal ? 1 : 2;
    const int lmax = kind == kTuneFinal ? 1 : L;
    if (level < lmin || level > lmax) return fail(PRNU_EINVAL, "level must be in [%d, %d] for this kind", lmin, lmax);
    if (choice < -2 || choice >= nch) return fail(PRNU_EINVAL, "choice must be in [-2, %d)", nch);
    std::lock_guard<std::mutex> lk(ctx->mu);
    const auto key = std::make_tuple(padded(H, L), padded(W, L), (int)params->dtype, kind, level);
    if (choice == -1)
        ctx->tuned_lv.erase(key);
    else if (choice >= 0)
        ctx->tuned_lv[key] = choice;
    if (current) {
        auto it = ctx->tuned_lv.find(key);
        *current = it == ctx->tuned_lv.end() ? 0 : it->second;
    }
    return PRNU_OK;
}

prnu_status prnu_autotune_set(prnu_ctx *ctx, int H, int W, const prnu_params *params, int shape) {
    if (!ctx) return fail(PRNU_EINVAL, "ctx is NULL");
    prnu_status s;
    if ((s = check_geometry(H, W, 1)) != PRNU_OK) return s;
    if ((s = check_params(params, H, W, nullptr)) != PRNU_OK) return s;
    if (shape < -1 || shape >= kStreamShapes) return fail(PRNU_EINVAL, "shape must be in [-1, %d)", kStreamShapes);
    const int L = params->levels;
    std::lock_guard<std::mutex> lk(ctx->mu);
    const auto key = std::make_tuple(padded(H, L), padded(W, L), (int)params->dtype);
    if (shape < 0) {
        ctx->tuned.erase(key);
        // the defaults for every level
        for (auto it = ctx->tuned_lv.begin(); it != ctx->tuned_lv.end();) {
            if (std::get<0>(it->first) == std::get<0>(key) && std::get<1>(it->first) == std::get<1>(key) &&
                std::get<2>(it->first) == std::get<2>(key))
                it = ctx->tuned_lv.erase(it);
            else
                ++it;
        }
    } else {
        ctx->tuned[key] = shape;
    }
    return PRNU_OK;
}

prnu_status prnu_debug_status(prnu_ctx *ctx, char *where, size_t where_len) {
    if (!ctx) return fail(PRNU_EINVAL, "ctx is NULL");
    if (where && where_len) where[0] = 0;
#ifndef PRNU_DEBUG
    return fail(PRNU_EUNSUPPORTED, "this library was built without PRNU_DEBUG (use libprnu_debug.so)");
#else
    DeviceGuard g(ctx->device);
    CU(cudaDeviceSynchronize());
    prnu_status st = PRNU_OK;
    for (auto &u : debug_registry()) {
        DebugWord w{0, 0, 0};
        CU(u.second(&w, true));
        if (w.hit && st == PRNU_OK) {
            const char *base = std::strrchr(u.first, '/');
            st = fail(PRNU_EDEBUG, "index check failed at %s:%d (index %lld)", base ? base + 1 : u.first, w.line,
                      w.index);
            if (where && where_len) snprintf(where, where_len, "%s:%d %lld", base ? base + 1 : u.first, w.line,
                                             w.index);
        }
    }
    return st;
#endif
}

prnu_status prnu_profile_enable(prnu_ctx *ctx, int on) {
    if (!ctx) return fail(PRNU_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->prof_on = on != 0;
    return PRNU_OK;
}

prnu_status prnu_profile_select(prnu_ctx *ctx, const char *names) {
    if (!ctx) return fail(PRNU_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->prof_sel.clear();
    for (const char *p = names; p && *p;) {
        const char *e = std::strchr(p, ',');
        const size_t len = e ? (size_t)(e - p) : std::strlen(p);
        if (len) ctx->prof_sel.emplace_back(p, len);
        p = e ? e + 1 : p + len;
    }
    return PRNU_OK;
}

prnu_status prnu_profile_reset(prnu_ctx *ctx) {
    if (!ctx) return fail(PRNU_EINVAL, "ctx is NULL");
    DeviceGuard g(ctx->device);
    std::lock_guard<std::mutex> lk(ctx->mu);
    for (auto &r : ctx->recs) {
        cudaEventSynchronize(r.b);
        ctx->pool.push_back(r.a);
        ctx->pool.push_back(r.b);
    }
    ctx->recs.clear();
    for (auto &n : ctx->klaunches) n = 0;
    for (auto &b : ctx->kbytes) b = 0.0;
    return PRNU_OK;
}

prnu_status prnu_profile_read(prnu_ctx *ctx, int index, char *name, size_t name_len, long long *launches,
                              double *total_ms, double *bytes) {
    if (!ctx) return fail(PRNU_EINVAL, "ctx is NULL");
    DeviceGuard g(ctx->device);
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (index < 0 || index >= (int)ctx->knames.size()) return fail(PRNU_EINVAL, "no kernel with index %d", index);
    if (name && name_len) {
        std::strncpy(name, ctx->knames[index].c_str(), name_len - 1);
        name[name_len - 1] = 0;
    }
    if (launches) *launches = ctx->klaunches[index];
    if (bytes) *bytes = ctx->kbytes[index];
    if (total_ms) {
        double t = 0.0;
        for (auto &r : ctx->recs) {
            if (r.kid != index) continue;
            float ms = 0.f;
            CU(cudaEventSynchronize(r.b));
            CU(cudaEventElapsedTime(&ms, r.a, r.b));
            t += ms;
        }
        *total_ms = t;
    }
    return PRNU_OK;
}

}  // extern "C"
