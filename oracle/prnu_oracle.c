/*
 * prnu_oracle.c -- plain FP64 CPU oracle for PRNU camera-fingerprint extraction
 * with Spatial Domain Averaged (SDA) frames (Taspinar, Mohanty, Memon,
 * "Camera Fingerprint Extraction via Spatial Domain Averaged Frames").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this file.  The product
 * path (the CUDA library) never calls it, and the two share no code.
 *
 * Every routine restates one step literally, in double precision, with no
 * blocking, fusion or reordering beyond what the definition states:
 *
 *   SDA frame (Sec. III-B, definition of I_i^SDA): mean of the frames of each
 *       disjoint group of d consecutive frames; a ragged last group is the mean
 *       of the frames it actually holds.
 *   Denoiser F (Sec. II-A / III-A cite the wavelet filter of Mihcak et al.;
 *       its parameters are the build's reading): L-level periodised orthonormal
 *       DWT with an 8-tap Daubechies lowpass h and highpass g[k]=(-1)^k h[7-k],
 *       a[n] = sum_k h[k] x[(2n+k) mod N], d[n] = sum_k g[k] x[(2n+k) mod N],
 *       rows first then columns; each detail coefficient c is shrunk with the
 *       minimum over the w x w windows (w in {3,5,7,9}, periodic wrap) of the
 *       mean of c^2: var = max(0, min_w mean_w - s0^2), clean = c var/(var+s0^2),
 *       noise = c s0^2/(var+s0^2); F(I) = IDWT(LL_L, clean details).
 *   Residual (Sec. II-A, W = I - F(I)) on the mirror-padded image, cropped.
 *   MLE (Sec. III-A equation for K-hat, and its SDA form in Sec. III-B):
 *       num += W.I, den += I.I accumulated over the frames (or SDA frames).
 *
 * Pins (tests/test_oracle_*.py) hold these loops to textbook values,
 * invariants and brute force; the exact denoiser output on natural-looking
 * content is held to an independent computation of the same definition
 * (explicit orthogonal level matrices from the published taps, a library box
 * filter for the window means, the transposed matrices for the inverse).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2

static long wrap_index(long i, long n)
{
    long r = i % n;
    return r < 0 ? r + n : r;
}

/* ------------------------------------------------------------------------ */
/* SDA frames, Sec. III-B: I_i^SDA = (1/n_i) sum of the frames of group i.   */
/* frames: uint8 [m][H][W][C] at byte offsets j*frame_stride + y*row_pitch  */
/* + x*C + c.  out: [g][C][H][W] doubles, g = ceil(m/d).                    */
/* ------------------------------------------------------------------------ */
int orc_sda_average(const uint8_t *frames, int m, int H, int W, int C,
                    long frame_stride, long row_pitch, int d, double *out)
{
    if (m < 1 || d < 1 || H < 1 || W < 1 || C < 1) return ORC_EINVAL;
    int g = (m + d - 1) / d;
    for (int i = 0; i < g; ++i) {
        int j0 = i * d;
        int j1 = (i + 1) * d < m ? (i + 1) * d : m;
        long n = j1 - j0;
        for (int c = 0; c < C; ++c) {
#pragma omp parallel for schedule(static)
            for (int y = 0; y < H; ++y) {
                for (int x = 0; x < W; ++x) {
                    long s = 0;
                    for (int j = j0; j < j1; ++j)
                        s += frames[(long)j * frame_stride + (long)y * row_pitch + (long)x * C + c];
                    out[(((long)i * C + c) * H + y) * W + x] = (double)s / (double)n;
                }
            }
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Mirror padding with edge repeat (..., x1, x0 | x0, x1, ...) on the high  */
/* side, so that both sides become multiples of 2^levels.                   */
/* ------------------------------------------------------------------------ */
static long mirror_index(long i, long n)
{
    /* i in [0, 2n): i < n maps to itself, i >= n maps to 2n-1-i */
    return i < n ? i : 2 * n - 1 - i;
}

int orc_pad_mirror(const double *img, int H, int W, int Hp, int Wp, double *out)
{
    if (Hp < H || Wp < W || Hp > 2 * H || Wp > 2 * W) return ORC_EINVAL;
    for (int y = 0; y < Hp; ++y)
        for (int x = 0; x < Wp; ++x)
            out[(long)y * Wp + x] = img[mirror_index(y, H) * W + mirror_index(x, W)];
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* One level of the periodised orthonormal 2-D DWT.                         */
/* ------------------------------------------------------------------------ */
static double highpass_tap(const double *h, int L, int k)
{
    /* g[k] = (-1)^k h[L-1-k] */
    return (k % 2 == 0 ? 1.0 : -1.0) * h[L - 1 - k];
}

/* a[n] = sum_k h[k] x[(2n+k) mod N],  b[n] = sum_k g[k] x[(2n+k) mod N] */
static void analysis_line(const double *x, long xs, int N, const double *h, int L,
                          double *a, double *b, long os)
{
    for (int n = 0; n < N / 2; ++n) {
        double lo = 0.0, hi = 0.0;
        for (int k = 0; k < L; ++k) {
            double v = x[wrap_index(2L * n + k, N) * xs];
            lo += h[k] * v;
            hi += highpass_tap(h, L, k) * v;
        }
        a[(long)n * os] = lo;
        b[(long)n * os] = hi;
    }
}

/* transpose of analysis_line: x[(2n+k) mod N] += h[k] a[n] + g[k] b[n] */
static void synthesis_line(const double *a, const double *b, long is, int N,
                           const double *h, int L, double *x, long xs)
{
    for (int j = 0; j < N; ++j) x[(long)j * xs] = 0.0;
    for (int n = 0; n < N / 2; ++n)
        for (int k = 0; k < L; ++k)
            x[wrap_index(2L * n + k, N) * xs] += h[k] * a[(long)n * is] + highpass_tap(h, L, k) * b[(long)n * is];
}

/* x: R x Cc (row-major).  Rows first (L/H along x), then columns.
 * LL = row-low/col-low, LH = row-low/col-high, HL = row-high/col-low,
 * HH = row-high/col-high; each (R/2) x (Cc/2). */
int orc_dwt2_level(const double *x, int R, int Cc, const double *h, int L,
                   double *LL, double *LH, double *HL, double *HH)
{
    if (R % 2 || Cc % 2 || R < 2 || Cc < 2) return ORC_EINVAL;
    int r2 = R / 2, c2 = Cc / 2;
    double *tl = (double *)malloc(sizeof(double) * (size_t)R * c2);
    double *th = (double *)malloc(sizeof(double) * (size_t)R * c2);
    if (!tl || !th) { free(tl); free(th); return ORC_ENOMEM; }
#pragma omp parallel for schedule(static)
    for (int r = 0; r < R; ++r)
        analysis_line(x + (long)r * Cc, 1, Cc, h, L, tl + (long)r * c2, th + (long)r * c2, 1);
#pragma omp parallel for schedule(static)
    for (int q = 0; q < c2; ++q) {
        analysis_line(tl + q, c2, R, h, L, LL + q, LH + q, c2);
        analysis_line(th + q, c2, R, h, L, HL + q, HH + q, c2);
    }
    free(tl);
    free(th);
    return ORC_OK;
}

/* Inverse of orc_dwt2_level: columns first, then rows.  x: R x Cc. */
int orc_idwt2_level(const double *LL, const double *LH, const double *HL, const double *HH,
                    int R, int Cc, const double *h, int L, double *x)
{
    if (R % 2 || Cc % 2 || R < 2 || Cc < 2) return ORC_EINVAL;
    int c2 = Cc / 2;
    double *tl = (double *)malloc(sizeof(double) * (size_t)R * c2);
    double *th = (double *)malloc(sizeof(double) * (size_t)R * c2);
    if (!tl || !th) { free(tl); free(th); return ORC_ENOMEM; }
#pragma omp parallel for schedule(static)
    for (int q = 0; q < c2; ++q) {
        synthesis_line(LL + q, LH + q, c2, R, h, L, tl + q, c2);
        synthesis_line(HL + q, HH + q, c2, R, h, L, th + q, c2);
    }
#pragma omp parallel for schedule(static)
    for (int r = 0; r < R; ++r)
        synthesis_line(tl + (long)r * c2, th + (long)r * c2, 1, Cc, h, L, x + (long)r * Cc, 1);
    free(tl);
    free(th);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Local-variance Wiener shrink of one detail subband (R x Cc).             */
/* mean_w = (1/w^2) sum over the w x w window centred on the coefficient,   */
/* indices wrapped periodically; v = min_w mean_w; var = max(0, v - s0^2).  */
/* noise = c s0^2/(var+s0^2), clean = c var/(var+s0^2) (both 0 when        */
/* var+s0^2 == 0, which forces c == 0).  Either output may be NULL.         */
/* ------------------------------------------------------------------------ */
int orc_shrink_subband(const double *c, int R, int Cc, double sigma0,
                       const int *windows, int n_windows,
                       double *noise, double *clean, double *var_out)
{
    if (n_windows < 1) return ORC_EINVAL;
    for (int i = 0; i < n_windows; ++i)
        if (windows[i] < 1 || windows[i] % 2 == 0) return ORC_EINVAL;
    double s2 = sigma0 * sigma0;
#pragma omp parallel for schedule(static)
    for (int r = 0; r < R; ++r) {
        for (int q = 0; q < Cc; ++q) {
            double vmin = INFINITY;
            for (int wi = 0; wi < n_windows; ++wi) {
                int w = windows[wi], rad = w / 2;
                double s = 0.0;
                for (int dy = -rad; dy <= rad; ++dy)
                    for (int dx = -rad; dx <= rad; ++dx) {
                        double v = c[wrap_index(r + dy, R) * Cc + wrap_index(q + dx, Cc)];
                        s += v * v;
                    }
                double mean = s / ((double)w * (double)w);
                if (mean < vmin) vmin = mean;
            }
            double var = vmin - s2 > 0.0 ? vmin - s2 : 0.0;
            double den = var + s2;
            double cv = c[(long)r * Cc + q];
            if (noise) noise[(long)r * Cc + q] = den > 0.0 ? cv * s2 / den : 0.0;
            if (clean) clean[(long)r * Cc + q] = den > 0.0 ? cv * var / den : 0.0;
            if (var_out) var_out[(long)r * Cc + q] = var;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Denoiser F on one padded plane (Hp x Wp, multiples of 2^levels).         */
/* F_out  = IDWT(LL_L, clean details)        (the denoised image F(I))      */
/* Wn_out = IDWT(0,    noise details)        (the noise form of I - F(I))   */
/* Either output may be NULL.                                               */
/* ------------------------------------------------------------------------ */
int orc_denoise_plane(const double *xp, int Hp, int Wp, int levels,
                      const double *h, int L, double sigma0,
                      const int *windows, int n_windows,
                      double *F_out, double *Wn_out)
{
    if (levels < 1 || levels > 8) return ORC_EINVAL;
    if (Hp % (1 << levels) || Wp % (1 << levels)) return ORC_EINVAL;
    int rc = ORC_OK;
    /* per level l = 1..levels: 4 subbands of (Hp>>l) x (Wp>>l) */
    double *LLs[9] = {0}, *D[9][3] = {{0}};
    double *cleanD[9][3] = {{0}}, *noiseD[9][3] = {{0}};
    double *rec = NULL, *recn = NULL, *tmp = NULL;
    for (int l = 1; l <= levels; ++l) {
        size_t n = (size_t)(Hp >> l) * (size_t)(Wp >> l);
        LLs[l] = (double *)malloc(n * sizeof(double));
        for (int s = 0; s < 3; ++s) {
            D[l][s] = (double *)malloc(n * sizeof(double));
            cleanD[l][s] = (double *)malloc(n * sizeof(double));
            noiseD[l][s] = (double *)malloc(n * sizeof(double));
            if (!D[l][s] || !cleanD[l][s] || !noiseD[l][s]) rc = ORC_ENOMEM;
        }
        if (!LLs[l]) rc = ORC_ENOMEM;
    }
    size_t np = (size_t)Hp * (size_t)Wp;
    rec = (double *)malloc(np * sizeof(double));
    recn = (double *)malloc(np * sizeof(double));
    tmp = (double *)malloc(np * sizeof(double));
    if (!rec || !recn || !tmp) rc = ORC_ENOMEM;
    if (rc != ORC_OK) goto done;

    /* analysis: level l acts on LL_{l-1} (LL_0 = the image) */
    for (int l = 1; l <= levels; ++l) {
        const double *src = l == 1 ? xp : LLs[l - 1];
        rc = orc_dwt2_level(src, Hp >> (l - 1), Wp >> (l - 1), h, L,
                            LLs[l], D[l][0], D[l][1], D[l][2]);
        if (rc) goto done;
        for (int s = 0; s < 3; ++s) {
            rc = orc_shrink_subband(D[l][s], Hp >> l, Wp >> l, sigma0, windows, n_windows,
                                    noiseD[l][s], cleanD[l][s], NULL);
            if (rc) goto done;
        }
    }
    /* synthesis, coarsest level first */
    {
        size_t n = (size_t)(Hp >> levels) * (size_t)(Wp >> levels);
        memcpy(rec, LLs[levels], n * sizeof(double));
        memset(recn, 0, n * sizeof(double));
    }
    for (int l = levels; l >= 1; --l) {
        int R = Hp >> (l - 1), Cc = Wp >> (l - 1);
        rc = orc_idwt2_level(rec, cleanD[l][0], cleanD[l][1], cleanD[l][2], R, Cc, h, L, tmp);
        if (rc) goto done;
        memcpy(rec, tmp, (size_t)R * Cc * sizeof(double));
        rc = orc_idwt2_level(recn, noiseD[l][0], noiseD[l][1], noiseD[l][2], R, Cc, h, L, tmp);
        if (rc) goto done;
        memcpy(recn, tmp, (size_t)R * Cc * sizeof(double));
    }
    if (F_out) memcpy(F_out, rec, np * sizeof(double));
    if (Wn_out) memcpy(Wn_out, recn, np * sizeof(double));
done:
    for (int l = 1; l <= levels; ++l) {
        free(LLs[l]);
        for (int s = 0; s < 3; ++s) { free(D[l][s]); free(cleanD[l][s]); free(noiseD[l][s]); }
    }
    free(rec);
    free(recn);
    free(tmp);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Noise residual of one plane, Sec. II-A: W = I - F(I).  img: H x W.      */
/* The plane is mirror-padded to Hp x Wp, denoised, subtracted, cropped.    */
/* ------------------------------------------------------------------------ */
int orc_residual_plane(const double *img, int H, int W, int levels,
                       const double *h, int L, double sigma0,
                       const int *windows, int n_windows, double *res)
{
    int m = 1 << levels;
    int Hp = (H + m - 1) / m * m, Wp = (W + m - 1) / m * m;
    double *xp = (double *)malloc(sizeof(double) * (size_t)Hp * Wp);
    double *F = (double *)malloc(sizeof(double) * (size_t)Hp * Wp);
    int rc = (!xp || !F) ? ORC_ENOMEM : ORC_OK;
    if (!rc) rc = orc_pad_mirror(img, H, W, Hp, Wp, xp);
    if (!rc) rc = orc_denoise_plane(xp, Hp, Wp, levels, h, L, sigma0, windows, n_windows, F, NULL);
    if (!rc)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x)
                res[(long)y * W + x] = img[(long)y * W + x] - F[(long)y * Wp + x];
    free(xp);
    free(F);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* MLE accumulation, Sec. III-A/III-B: num += W.I, den += I.I (elementwise).  */
/* ------------------------------------------------------------------------ */
void orc_mle_accumulate(const double *Wr, const double *I, long n, double *num, double *den)
{
    for (long i = 0; i < n; ++i) {
        num[i] += Wr[i] * I[i];
        den[i] += I[i] * I[i];
    }
}

/* K = num/den, 0 where den == 0 */
void orc_mle_finalize(const double *num, const double *den, long n, double *K)
{
    for (long i = 0; i < n; ++i) K[i] = den[i] != 0.0 ? num[i] / den[i] : 0.0;
}
