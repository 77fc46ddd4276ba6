// prnu_grad.cu -- entry points of the differentiable chain (prnu.h, section
// "Differentiation"): weighted SDA frames, the residual with its detail
// coefficients kept as a checkpoint, the MLE fingerprint of n residual/image
// pairs, and the adjoint of each step.
#include <cmath>

#include "abi_internal.cuh"

using namespace prnu;
using namespace prnu::abi;

namespace {

prnu_status check_grad_geometry(int H, int W, int C, const prnu_params *params, Win *win) {
    prnu_status s;
    if ((s = check_geometry(H, W, C)) != PRNU_OK) return s;
    if ((s = check_params(params, H, W, win)) != PRNU_OK) return s;
    if (params->dtype != PRNU_DTYPE_F32) return fail(PRNU_EUNSUPPORTED, "gradients need float32 subbands");
    const int m = 1 << params->levels;
    if (H % m || W % m)
        return fail(PRNU_EUNSUPPORTED, "gradients need H, W multiples of 2^levels = %d (got %d x %d)", m, H, W);
    return PRNU_OK;
}

size_t ckpt_floats(int H, int W, long long P, int L) {
    size_t n = 0;
    for (int l = 1; l <= L; ++l) n += (size_t)3 * P * (size_t)(H >> l) * (size_t)(W >> l);
    return n;
}

struct PceBwdLayout {
    size_t real0 = 0, real1 = 0, cplx0 = 0, cplx1 = 0;
    size_t pm = 0, pe = 0, pv = 0, pi = 0, scal = 0, work = 0, end = 0;
    int nb = 0;
};

prnu_status pce_bwd_layout(prnu_ctx *ctx, int H, int W, int n, PceBwdLayout *out) {
    PceBwdLayout f;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, kAlign);
        return o;
    };
    const size_t hw = (size_t)H * W, nh = (size_t)H * (W / 2 + 1);
    f.nb = (int)std::min<size_t>(256, std::max<size_t>(1, hw / (256 * 16)));
    f.real0 = take(2 * (size_t)n * hw * sizeof(float));
    f.real1 = take((size_t)n * hw * sizeof(float));
    f.cplx0 = take(2 * (size_t)n * nh * sizeof(cufftComplex));
    f.cplx1 = take((size_t)n * nh * sizeof(cufftComplex));
    f.pm = take((size_t)n * f.nb * 4 * sizeof(double));
    f.pe = take((size_t)n * f.nb * sizeof(double));
    f.pv = take((size_t)n * f.nb * sizeof(float));
    f.pi = take((size_t)n * f.nb * sizeof(long long));
    f.scal = take((size_t)n * pce_scalars_bytes());
    size_t w = 0, wmax = 0;
    cufftHandle p;
    prnu_status s;
    const cufftType types[4] = {CUFFT_R2C, CUFFT_C2R, CUFFT_R2C, CUFFT_C2R};
    const int batches[4] = {2 * n, n, n, 2 * n};
    for (int i = 0; i < 4; ++i) {
        if ((s = get_plan(ctx, H, W, types[i], batches[i], &p, &w)) != PRNU_OK) return s;
        wmax = std::max(wmax, w);
    }
    f.work = take(wmax);
    f.end = off;
    *out = f;
    return PRNU_OK;
}

}  // namespace

extern "C" {

prnu_status prnu_sda_weighted(prnu_ctx *ctx, const uint8_t *frames, int m, int H, int W, int C, size_t frame_stride,
                              size_t row_pitch, int d, const float *weights, float *sda_out, void *stream) {
    if (!ctx || !frames || !weights || !sda_out) return fail(PRNU_EINVAL, "NULL argument");
    prnu_status s;
    if ((s = check_geometry(H, W, C)) != PRNU_OK) return s;
    if (m < 1 || d < 1 || d > m) return fail(PRNU_EINVAL, "need 1 <= d <= m (d=%d, m=%d)", d, m);
    if (row_pitch < (size_t)W * C) return fail(PRNU_EINVAL, "row_pitch < W*C");
    if (m > 1 && frame_stride < (size_t)(H - 1) * row_pitch + (size_t)W * C)
        return fail(PRNU_EINVAL, "frame_stride too small");
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
    a.G = (m + d - 1) / d;
    a.out = sda_out;
    Launch t(ctx, "sda_weighted", S(stream), 1, (double)m * H * W * C + (double)a.G * C * H * W * 4);
    CU(launch_sda_weighted(a, weights, ctx->sms, S(stream)));
    return PRNU_OK;
}

prnu_status prnu_sda_weighted_backward(prnu_ctx *ctx, const uint8_t *frames, int m, int H, int W, int C,
                                       size_t frame_stride, size_t row_pitch, int d, const float *g_sda,
                                       float *g_weights, void *ws, size_t ws_bytes, void *stream) {
    if (!ctx || !frames || !g_sda || !g_weights) return fail(PRNU_EINVAL, "NULL argument");
    prnu_status s;
    if ((s = check_geometry(H, W, C)) != PRNU_OK) return s;
    if (m < 1 || d < 1 || d > m) return fail(PRNU_EINVAL, "need 1 <= d <= m (d=%d, m=%d)", d, m);
    if (row_pitch < (size_t)W * C) return fail(PRNU_EINVAL, "row_pitch < W*C");
    if (m > 1 && frame_stride < (size_t)(H - 1) * row_pitch + (size_t)W * C)
        return fail(PRNU_EINVAL, "frame_stride too small");
    if ((s = check_ws(ws, ws_bytes, (size_t)m * sda_wgrad_blocks(H) * sizeof(double))) != PRNU_OK) return s;
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
    Launch t(ctx, "sda_weighted_bwd", S(stream), 2, (double)m * H * W * C * 5);
    CU(launch_sda_wgrad(a, g_sda, static_cast<double *>(ws), g_weights, S(stream)));
    return PRNU_OK;
}

prnu_status prnu_workspace_size_grad(prnu_ctx *ctx, int H, int W, int C, const prnu_params *params, int n,
                                     size_t *ws_bytes, size_t *ckpt_bytes) {
    if (!ctx || !ws_bytes || !ckpt_bytes) return fail(PRNU_EINVAL, "NULL argument");
    if (n < 1) return fail(PRNU_EINVAL, "n must be >= 1");
    prnu_status s;
    if ((s = check_grad_geometry(H, W, C, params, nullptr)) != PRNU_OK) return s;
    *ws_bytes = make_layout(H, W, (long long)n * C, params->levels, false, PRNU_DTYPE_F32).end;
    *ckpt_bytes = ckpt_floats(H, W, (long long)n * C, params->levels) * sizeof(float);
    return PRNU_OK;
}

prnu_status prnu_denoise_residual_ckpt(prnu_ctx *ctx, const float *img, int n, int H, int W, int C,
                                       const prnu_params *params, float *residual_out, float *ckpt, void *ws,
                                       size_t ws_bytes, void *stream) {
    if (!ctx || !img || !residual_out || !ckpt) return fail(PRNU_EINVAL, "NULL argument");
    if ((const void *)img == (const void *)residual_out) return fail(PRNU_EINVAL, "img and residual_out alias");
    if (n < 1) return fail(PRNU_EINVAL, "n must be >= 1");
    prnu_status s;
    Win win;
    if ((s = check_grad_geometry(H, W, C, params, &win)) != PRNU_OK) return s;
    const long long P = (long long)n * C;
    const Layout lo = make_layout(H, W, P, params->levels, false, PRNU_DTYPE_F32);
    if ((s = check_ws(ws, ws_bytes, lo.end)) != PRNU_OK) return s;
    DeviceGuard g(ctx->device);
    cudaStream_t st = S(stream);
    FinalArgs fin{};
    fin.C = C;
    fin.G = n;
    fin.res_out = residual_out;
    fin.sc = PlaneScale{1, 1, 0, C, nullptr};
    if ((s = run_denoise(ctx, img, H, W, (int)P, *params, win, fin.sc, 0, static_cast<char *>(ws), lo, fin, false,
                         st)) != PRNU_OK)
        return s;
    // the checkpoint: every level's detail coefficients, level after level
    size_t off = 0;
    for (int l = 1; l <= params->levels; ++l) {
        const size_t bytes = (size_t)3 * P * (size_t)(H >> l) * (size_t)(W >> l) * sizeof(float);
        CU(cudaMemcpyAsync(reinterpret_cast<char *>(ckpt) + off, static_cast<char *>(ws) + lo.D[l], bytes,
                           cudaMemcpyDeviceToDevice, st));
        off += bytes;
    }
    return PRNU_OK;
}

prnu_status prnu_denoise_residual_backward(prnu_ctx *ctx, const float *ckpt, int n, int H, int W, int C,
                                           const prnu_params *params, const float *g_residual, float *g_img,
                                           double *g_sigma0, void *ws, size_t ws_bytes, void *stream) {
    if (!ctx || !ckpt || !g_residual || !g_img) return fail(PRNU_EINVAL, "NULL argument");
    if ((const void *)g_residual == (const void *)g_img) return fail(PRNU_EINVAL, "g_residual and g_img alias");
    if (n < 1) return fail(PRNU_EINVAL, "n must be >= 1");
    prnu_status s;
    Win win;
    if ((s = check_grad_geometry(H, W, C, params, &win)) != PRNU_OK) return s;
    const long long P = (long long)n * C;
    const Layout lo = make_layout(H, W, P, params->levels, false, PRNU_DTYPE_F32);
    if ((s = check_ws(ws, ws_bytes, lo.end)) != PRNU_OK) return s;
    DeviceGuard g(ctx->device);
    FinalArgs fin{};
    fin.C = C;
    fin.G = n;
    fin.res_out = g_img;
    fin.accumulate = 1;
    fin.sc = PlaneScale{1, 1, 0, C, nullptr};
    return run_denoise(ctx, g_residual, H, W, (int)P, *params, win, fin.sc, 0, static_cast<char *>(ws), lo, fin,
                       false, S(stream), ckpt, g_sigma0);
}

prnu_status prnu_mle_images(prnu_ctx *ctx, const float *residual, const float *img, int n, int H, int W, int C,
                            int gray, float *num, float *den, float *K, void *stream) {
    if (!ctx || !residual || !img || !num || !den || !K) return fail(PRNU_EINVAL, "NULL argument");
    if (n < 1) return fail(PRNU_EINVAL, "n must be >= 1");
    prnu_status s;
    if ((s = check_geometry(H, W, C)) != PRNU_OK) return s;
    if (gray != 0 && gray != 1) return fail(PRNU_EINVAL, "gray must be 0 or 1");
    DeviceGuard g(ctx->device);
    const long long hw = (long long)H * W;
    Launch t(ctx, "mle_images", S(stream), 1, (double)n * C * hw * 8 + (double)C * hw * 8 + (gray ? 1 : C) * hw * 4.0);
    CU(launch_mle_images(residual, img, n, C, hw, gray, num, den, K, ctx->sms, S(stream)));
    return PRNU_OK;
}

prnu_status prnu_mle_images_backward(prnu_ctx *ctx, const float *residual, const float *img, int n, int H, int W,
                                     int C, int gray, const float *num, const float *den, const float *g_K,
                                     float *g_residual, float *g_img, void *stream) {
    if (!ctx || !residual || !img || !num || !den || !g_K || !g_residual || !g_img)
        return fail(PRNU_EINVAL, "NULL argument");
    if (n < 1) return fail(PRNU_EINVAL, "n must be >= 1");
    prnu_status s;
    if ((s = check_geometry(H, W, C)) != PRNU_OK) return s;
    if (gray != 0 && gray != 1) return fail(PRNU_EINVAL, "gray must be 0 or 1");
    DeviceGuard g(ctx->device);
    const long long hw = (long long)H * W;
    Launch t(ctx, "mle_images_bwd", S(stream), 1, (double)n * C * hw * 16 + (double)C * hw * 12);
    CU(launch_mle_images_bwd(residual, img, n, C, hw, gray, num, den, g_K, g_residual, g_img, ctx->sms, S(stream)));
    return PRNU_OK;
}

prnu_status prnu_workspace_size_pce_backward(prnu_ctx *ctx, int H, int W, int n, size_t *bytes) {
    if (!ctx || !bytes) return fail(PRNU_EINVAL, "NULL argument");
    if (n < 1) return fail(PRNU_EINVAL, "n must be >= 1");
    prnu_status s;
    if ((s = check_geometry(H, W, 1)) != PRNU_OK) return s;
    DeviceGuard g(ctx->device);
    PceBwdLayout f;
    if ((s = pce_bwd_layout(ctx, H, W, n, &f)) != PRNU_OK) return s;
    *bytes = f.end;
    return PRNU_OK;
}

prnu_status prnu_pce_backward(prnu_ctx *ctx, const float *K, int per_query, const float *residual_q, const float *img_q,
                              int n, int H, int W, int C, int nbhd, const double *g_pce, float *g_K,
                              float *g_residual_q, void *ws, size_t ws_bytes, void *stream) {
    if (!ctx || !K || !residual_q || !img_q || !g_pce || !g_K || !g_residual_q)
        return fail(PRNU_EINVAL, "NULL argument");
    if (n < 1) return fail(PRNU_EINVAL, "n must be >= 1");
    if (per_query != 0 && per_query != 1) return fail(PRNU_EINVAL, "per_query must be 0 or 1");
    prnu_status s;
    if ((s = check_geometry(H, W, C)) != PRNU_OK) return s;
    if (nbhd < 1 || nbhd % 2 == 0 || nbhd > H || nbhd > W) return fail(PRNU_EINVAL, "nbhd must be odd and <= min(H, W)");
    DeviceGuard g(ctx->device);
    PceBwdLayout f;
    if ((s = pce_bwd_layout(ctx, H, W, n, &f)) != PRNU_OK) return s;
    if ((s = check_ws(ws, ws_bytes, f.end)) != PRNU_OK) return s;
    cudaStream_t st = S(stream);
    char *b = static_cast<char *>(ws);
    const long long hw = (long long)H * W, nh = (long long)H * (W / 2 + 1);
    float *X = reinterpret_cast<float *>(b + f.real0);  // X_0..X_{n-1}, Y_0..Y_{n-1}
    float *Cr = reinterpret_cast<float *>(b + f.real1);
    cufftComplex *FX = reinterpret_cast<cufftComplex *>(b + f.cplx0), *FY = FX + n * nh;
    cufftComplex *Z = reinterpret_cast<cufftComplex *>(b + f.cplx1);
    cufftHandle r2c2, c2r1, r2c1, c2r2;
    size_t w;
    if ((s = get_plan(ctx, H, W, CUFFT_R2C, 2 * n, &r2c2, &w)) != PRNU_OK) return s;
    if ((s = get_plan(ctx, H, W, CUFFT_C2R, n, &c2r1, &w)) != PRNU_OK) return s;
    if ((s = get_plan(ctx, H, W, CUFFT_R2C, n, &r2c1, &w)) != PRNU_OK) return s;
    if ((s = get_plan(ctx, H, W, CUFFT_C2R, 2 * n, &c2r2, &w)) != PRNU_OK) return s;
    {  // forward recomputation: X = grey(W_q), Y = K grey(I_q), C = corr(X, Y)
        Launch t(ctx, "pce_prep", st, 1, (double)n * hw * 4 * (2 * C + 2) + (double)hw * 4);
        CU(launch_pce_prep(K, per_query ? hw : 0, residual_q, img_q, hw, C, n, f.nb, X, X + n * hw,
                           reinterpret_cast<double *>(b + f.pm), st));
    }
    auto exec = [&](cufftHandle p, const char *name, bool r2c, void *in, void *out) -> prnu_status {
        Launch t(ctx, name, st);
        CUFFT(cufftSetStream(p, st));
        CUFFT(cufftSetWorkArea(p, b + f.work));
        if (r2c)
            CUFFT(cufftExecR2C(p, static_cast<cufftReal *>(in), static_cast<cufftComplex *>(out)));
        else
            CUFFT(cufftExecC2R(p, static_cast<cufftComplex *>(in), static_cast<cufftReal *>(out)));
        return PRNU_OK;
    };
    if ((s = exec(r2c2, "cufft_r2c", true, X, FX)) != PRNU_OK) return s;
    {
        Launch t(ctx, "pce_cross_spectrum", st, 1, (double)n * nh * 24);
        CU(launch_cross_spectrum(FX, FY, nh, n, Z, ctx->sms, st));
    }
    if ((s = exec(c2r1, "cufft_c2r", false, Z, Cr)) != PRNU_OK) return s;
    {
        Launch t(ctx, "pce_reduce", st, 2, (double)n * hw * 4);
        CU(launch_pce_reduce(Cr, H, W, nbhd / 2, n, f.nb, reinterpret_cast<double *>(b + f.pe),
                             reinterpret_cast<float *>(b + f.pv), reinterpret_cast<long long *>(b + f.pi),
                             reinterpret_cast<double *>(b + f.pm), f.nb, b + f.scal, st));
    }
    {  // adjoint: G = dPCE/dC, then a correlation with Y and a convolution with X
        Launch t(ctx, "pce_gfield", st, 1, (double)n * hw * 8);
        CU(launch_pce_gfield(Cr, H, W, nbhd / 2, n, b + f.scal, g_pce, st));
    }
    if ((s = exec(r2c1, "cufft_r2c", true, Cr, Z)) != PRNU_OK) return s;
    {
        Launch t(ctx, "pce_spectra_bwd", st, 1, (double)n * nh * 40);
        CU(launch_pce_spectra_bwd(FX, FY, Z, nh, n, ctx->sms, st));
    }
    if ((s = exec(c2r2, "cufft_c2r", false, FX, X)) != PRNU_OK) return s;  // X: N gY (n planes), N gX (n planes)
    {
        Launch t(ctx, "pce_bwd_out", st, 1, (double)n * hw * 4 * (2 + 2 * C) + (double)(per_query ? n : 1) * hw * 4);
        CU(launch_pce_bwd_out(X, X + n * hw, img_q, n, C, hw, (float)(1.0 / (double)hw), per_query, g_K, g_residual_q,
                              ctx->sms, st));
    }
    return PRNU_OK;
}

}  // extern "C"
