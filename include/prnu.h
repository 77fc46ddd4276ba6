/*
 * prnu.h -- C ABI of libprnu: GB300 (sm_103a) kernels for PRNU camera-
 * fingerprint extraction with Spatial Domain Averaged (SDA) frames
 * (Taspinar, Mohanty, Memon, "Camera Fingerprint Extraction via Spatial
 * Domain Averaged Frames").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named as device pointers must point to device memory of the
 *   context's device; the caller owns every buffer.  Entry points that take a
 *   workspace (`ws`, `ws_bytes`) use only that memory for intermediates and
 *   call no allocator, except that cuFFT plans are created (and cached in the
 *   context) on the first FFT of a given size: make that first call before
 *   any stream capture.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   All work is enqueued asynchronously on it, except prnu_pce_match, which
 *   synchronises the stream to return its scalars in host memory.
 * - Arguments are validated on the host before any launch.  Invalid input
 *   returns PRNU_EINVAL and launches nothing; a workspace that is too small
 *   returns PRNU_ENOSPC.  A CUDA or cuFFT failure returns PRNU_ECUDA.  The
 *   message of the last failure on the calling thread is returned by
 *   prnu_last_error().  No C++ exception crosses this interface.
 * - Images are planar float32 [C][H][W] in 0..255 units unless stated; frames
 *   are uint8 interleaved [m][H][W][C] at byte offset
 *   j*frame_stride + y*row_pitch + x*C + c.
 * - Limits: 16 <= H, W; H, W <= 16384; C in {1, 3}; 1 <= levels <= 6 with
 *   H, W >= 2^levels; windows odd in [1, 9]; 1 <= d <= m; d <= 65793 (so that
 *   a group sum of uint8 frames is an exact float32 integer).
 */
#ifndef PRNU_H
#define PRNU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PRNU_OK = 0,
    PRNU_EINVAL = -1,      /* invalid argument (nothing launched) */
    PRNU_ENOSPC = -2,      /* workspace too small (nothing launched) */
    PRNU_ECUDA = -3,       /* CUDA runtime or cuFFT error */
    PRNU_ETIMEOUT = -4,    /* a bounded device-side wait gave up */
    PRNU_EUNSUPPORTED = -5, /* valid but not implemented (e.g. dtype) */
    PRNU_EDEBUG = -6        /* debug build: a device-side index check failed */
} prnu_status;

/* Flags of prnu_fingerprint_finalize. */
#define PRNU_ZERO_MEAN 1u  /* subtract column means, then row means, per plane */
#define PRNU_WIENER_DFT 2u /* Wiener shrink of |DFT|/sqrt(N) with var(K) noise */
#define PRNU_TO_GRAY 4u    /* 0.299 R + 0.587 G + 0.114 B before the above */

/* Storage of the intermediate detail / noise subbands (arithmetic is always
 * float32; the lowpass chain is always a float32 float-float pair). */
#define PRNU_DTYPE_F32 0
#define PRNU_DTYPE_F16 1
#define PRNU_DTYPE_BF16 2
/* Element type of the input frames of the accumulate calls. */
#define PRNU_FRAMES_U8 0
#define PRNU_FRAMES_F16 1

/* Denoiser parameters.  The paper names the wavelet denoiser of Mihcak et
 * al. only by citation (Sec. III-A, Sec. IV); these are the build's reading:
 * orthonormal periodised 8-tap Daubechies DWT, `levels` levels, local
 * variance = min over the odd windows of the periodic box mean of c^2,
 * var = max(0, min - sigma0^2), noise coefficient c*sigma0^2/(var+sigma0^2). */
typedef struct {
    int levels;      /* 4 */
    float sigma0;    /* 3.0, in 0..255 pixel units; >= 0 */
    int n_windows;   /* 4 */
    int windows[4];  /* 3, 5, 7, 9 */
    int pad_mode;    /* 0 = mirror with edge repeat to multiples of 2^levels */
    int dtype;       /* subband storage: PRNU_DTYPE_F32 (default), _F16 or _BF16 */
    int frame_dtype; /* accumulate input frames: PRNU_FRAMES_U8 (default) or _F16 (values in 0..255 units;
                        frame_stride and row_pitch stay in bytes) */
    int compensated; /* 0: num/den are float32 [C][H][W];  1: compensated sums, num and den each point to
                        [2][C][H][W] float32 (the float-float pair hi, then lo, both zero-initialised by the
                        caller), accumulated with TwoSum error terms; finalize then reads both parts */
    int sda_blocks_per_sm; /* 0 (default): the SDA group-sum kernel fills every SM (2 blocks per SM when it
                              reads page-locked host frames); 1..32: at most that many of its blocks per SM,
                              leaving room for kernels that run concurrently on other streams (e.g.
                              prnu_pce_images_prepare or a pipelined accumulate's denoising) */
    int pipeline_passes;   /* prnu_fingerprint_accumulate with device frames: 0 or 1 (default): one stream,
                              each pass's group sums then its denoising; n >= 2: the groups are split into n
                              passes (or more, if two pass layouts of ceil(groups/n) groups do not fit the
                              workspace) and the group sums of pass k+1 run on the context's side stream while
                              pass k is denoised on `stream` (two pass layouts in the workspace; the sums kernel
                              then takes at most sda_blocks_per_sm blocks per SM, 6 when that is 0) */
    int sda_fusion;        /* the group sums and their level-1 analysis as one kernel (Sec. III-B averaging +
                              the first DWT level; the SDA frame still goes to the workspace for the MLE step)
                              where that applies -- uint8 frames, C = 1 or 3, W a multiple of 2^levels with
                              W*C a multiple of 16, 16-byte aligned frames and strides, groups of at most 257
                              frames -- else the separate kernels.  0 (default): fused in
                              prnu_fingerprint_accumulate with device frames (one stream) for d >= 16 and in
                              a pass of prnu_fingerprint_accumulate_multi whose groups average 16 frames or
                              more, separate for shorter groups; PRNU_SDA_SEPARATE: always separate;
                              PRNU_SDA_FUSED: fused in both wherever it applies, row strips chosen per launch;
                              n >= 1 (at most 256): the same with n row strips per column */
} prnu_params;
#define PRNU_SDA_SEPARATE (-1)
#define PRNU_SDA_FUSED (-2)

typedef struct prnu_ctx prnu_ctx; /* opaque; owns no per-call buffers */

/* Fill *p with the defaults above.  Never fails for non-NULL p. */
prnu_status prnu_default_params(prnu_params *p);

/* Create a context on CUDA device `device`: derives the filter bank (passed
 * to the kernels as launch parameters), creates a copy stream and events for
 * prnu_fingerprint_accumulate_host.  *out is NULL on failure. */
prnu_status prnu_create(prnu_ctx **out, int device);

/* Destroy a context (NULL allowed).  The caller must have synchronised every
 * stream that still runs work enqueued through it. */
void prnu_destroy(prnu_ctx *ctx);

/* Message of the last failure on the calling thread ("" if none).  The
 * pointer stays valid until the next call on this thread. */
const char *prnu_last_error(const prnu_ctx *ctx);

/* Bytes of workspace needed, for an H x W x C geometry, by
 * prnu_denoise_residual_batch and prnu_pce_match_batch with n <=
 * images_per_pass, by prnu_fingerprint_accumulate running up to
 * images_per_pass SDA frames (frames when d = 1) per pass (a larger workspace
 * means fewer passes), and by prnu_fingerprint_finalize.  Creates the cuFFT
 * plans of that size and batch in the context. */
prnu_status prnu_workspace_size(prnu_ctx *ctx, int H, int W, int C, const prnu_params *params,
                                int images_per_pass, size_t *bytes);

/* Bytes of workspace needed by prnu_fingerprint_accumulate_host for groups
 * of d frames with groups_per_pass groups copied per chunk (two staging
 * buffers of groups_per_pass*d packed frames plus the pass intermediates). */
prnu_status prnu_workspace_size_host(prnu_ctx *ctx, int H, int W, int C, int d, const prnu_params *params,
                                     int groups_per_pass, size_t *bytes);

/* SDA frames, Sec. III-B (definition of I_i^SDA): group i holds frames
 * i*d .. min((i+1)*d, m)-1 and its SDA frame is their arithmetic mean (a
 * ragged last group is the mean of the frames it holds).
 * frames: device uint8 [m][H][W][C] (strides in bytes).
 * sda_out: device float32 [ceil(m/d)][C][H][W], each value the correctly
 * rounded float32 of the exact mean. */
prnu_status prnu_sda_average(prnu_ctx *ctx, const uint8_t *frames, int m, int H, int W, int C,
                             size_t frame_stride, size_t row_pitch, int d, float *sda_out, void *stream);

/* Noise residual, Sec. II-A: W = I - F(I), with F the wavelet denoiser of
 * `params`, computed as the inverse DWT of the shrunk-away (noise) detail
 * coefficients of the mirror-padded image, cropped back to H x W.
 * img, residual_out: device float32 [C][H][W] (may not alias). */
prnu_status prnu_denoise_residual(prnu_ctx *ctx, const float *img, int H, int W, int C,
                                  const prnu_params *params, float *residual_out,
                                  void *ws, size_t ws_bytes, void *stream);

/* Batched residuals, Sec. II-A: n independent images img [n][C][H][W] ->
 * residual_out [n][C][H][W] in one pass of the kernels (same semantics as n
 * calls of prnu_denoise_residual). */
prnu_status prnu_denoise_residual_batch(prnu_ctx *ctx, const float *img, int n, int H, int W, int C,
                                        const prnu_params *params, float *residual_out,
                                        void *ws, size_t ws_bytes, void *stream);

/* Allocation-free variant of prnu_denoise_residual (the paper has no
 * counterpart: this is an interface convenience).  For callers that cannot
 * allocate device memory when they need a residual -- code running inside a
 * CUDA stream capture, plug-ins whose host application owns every device
 * allocation, services that fix their memory footprint at start-up -- the
 * intermediates live in a fixed 64 MiB file-scope device array of the library
 * instead of a caller workspace.  The caller still passes img and
 * residual_out (same layout and meaning as prnu_denoise_residual).  The
 * arguments are validated first, exactly as prnu_denoise_residual does
 * (EINVAL, nothing resolved or launched).  Images whose intermediates exceed
 * 64 MiB return PRNU_ENOSPC with a message and launch nothing; the need
 * depends on the subband type: with float32 subbands 1920x1080 grey and
 * 1280x720 RGB fit and 1920x1080 RGB does not, with float16 / bfloat16
 * subbands 1920x1080 RGB fits.  The first call with each context resolves the
 * array's device address on the context's device (cudaGetSymbolAddress,
 * which loads the module that holds the array) and keeps it in the context:
 * make that first call before any stream capture (a context created after a
 * device reset resolves it again).  Every GPU on which the array's module is
 * loaded keeps the 64 MiB until the process exits.  All calls on a device
 * share the array: calls whose GPU work may overlap (other streams or threads
 * without ordering) race and corrupt each other's results; calls ordered on
 * one stream are safe, and no clearing is needed between them. */
prnu_status prnu_denoise_residual_static(prnu_ctx *ctx, const float *img, int H, int W, int C,
                                         const prnu_params *params, float *residual_out, void *stream);

/* MLE fingerprint sums, Sec. III-A (K-hat = sum W_i I_i / sum I_i^2) over
 * the SDA frames of Sec. III-B (d = 1 is the conventional per-frame
 * estimator): for every group i, I_i = its SDA frame, W_i = I_i - F(I_i), and
 *     num += W_i * I_i,   den += I_i * I_i   (elementwise, per channel).
 * frames: device uint8 [m][H][W][C]; num, den: device float32 [C][H][W],
 * caller-initialised (zero to start); calls accumulate, so a long sequence
 * may be fed in pieces whose lengths are multiples of d (checkpoint = the
 * pair num/den plus the count of frames consumed). */
prnu_status prnu_fingerprint_accumulate(prnu_ctx *ctx, const uint8_t *frames, int m, int H, int W, int C,
                                        size_t frame_stride, size_t row_pitch, int d,
                                        const prnu_params *params, float *num, float *den,
                                        void *ws, size_t ws_bytes, void *stream);

/* Same as prnu_fingerprint_accumulate, but `host_frames` is host memory.
 * Page-locked frames (cudaHostAlloc / cudaHostRegister) are read in place by
 * the kernels through their device-visible address (no staging copy; the
 * whole workspace holds pass intermediates).  Pageable frames are copied in
 * chunks through two staging buffers in the workspace, each copy overlapping
 * the kernels of the previous chunk.  Either way the frames must stay
 * unchanged until the stream has run the work.  num, den are device
 * pointers. */
prnu_status prnu_fingerprint_accumulate_host(prnu_ctx *ctx, const uint8_t *host_frames, int m, int H, int W,
                                             int C, size_t frame_stride, size_t row_pitch, int d,
                                             const prnu_params *params, float *num, float *den,
                                             void *ws, size_t ws_bytes, void *stream);

/* One camera of a multi-camera batch: its frames (device; uint8 or float16 per
 * params->frame_dtype), frame count, geometry, byte strides, SDA group size
 * (ragged last group) and its own MLE sums (device float32 [C][H][W], or
 * [2][C][H][W] with params->compensated; accumulated into, as for
 * prnu_fingerprint_accumulate).  Cameras must not share num/den. */
typedef struct {
    const uint8_t *frames;
    int m, H, W, C;
    size_t frame_stride, row_pitch;
    int d;
    float *num, *den;
} prnu_camera;

/* Workspace for prnu_fingerprint_accumulate_multi running up to
 * groups_per_pass SDA groups (1..192) of one geometry per pass. */
prnu_status prnu_workspace_size_multi(prnu_ctx *ctx, const prnu_camera *cams, int ncams, const prnu_params *params,
                                      int groups_per_pass, size_t *bytes);

/* MLE fingerprint sums (Sec. III-A / III-B) of many cameras with uneven frame
 * counts, resolutions and SDA group sizes in one call: cameras are grouped by
 * geometry and their groups packed into passes that mix cameras (each pass is
 * one launch of every kernel of the pipeline, with a per-group table of frame
 * pointers, counts and destination camera).  `cams` is a host array.  Same
 * results as one prnu_fingerprint_accumulate per camera.  Allocates nothing,
 * synchronises nothing: the call can be captured in a CUDA graph once the
 * workspace exists. */
prnu_status prnu_fingerprint_accumulate_multi(prnu_ctx *ctx, const prnu_camera *cams, int ncams,
                                              const prnu_params *params, void *ws, size_t ws_bytes, void *stream);

/* The MLE sums of prnu_fingerprint_accumulate_multi (Sec. III-A over the SDA
 * frames of Sec. III-B, many cameras of uneven frame counts, resolutions and
 * group sizes) in ONE persistent kernel launch.  Every block of the launch
 * claims items from a device work queue -- one tile of one stage (SDA sums,
 * analysis of a level, shrink of a level, synthesis of a level, level-1
 * synthesis with the MLE sums) of one SDA group -- waits until the stages the
 * item reads have completed, runs it and counts it.  The host orders the
 * queue so that the frame reads of one group run beside the denoising of the
 * two groups before it.  A group's intermediates live in one of `slots`
 * workspace slots (3..64; a slot is reused by group g + slots once group g's
 * MLE step is done); each camera's groups are added to its num/den one at a
 * time, in order.  Every device-side wait gives up after wait_budget_ms
 * (0 = 2000 ms) of the GPU's global timer: the launch then records
 * PRNU_ETIMEOUT and the failing item in the workspace and ends without
 * completing the sums; prnu_persistent_status reports it.  uint8 frames and
 * float32 subbands (PRNU_EUNSUPPORTED otherwise); num/den as in
 * prnu_fingerprint_accumulate (float32 [C][H][W], or compensated pairs).
 * Same results as prnu_fingerprint_accumulate_multi up to the order of the
 * float32 MLE additions.  Allocates nothing and synchronises nothing (one
 * memset, a few small copy kernels and the persistent kernel), so the call can
 * be captured in a CUDA graph; at most 8 distinct geometries per call. */
prnu_status prnu_workspace_size_persistent(prnu_ctx *ctx, const prnu_camera *cams, int ncams,
                                           const prnu_params *params, int slots, size_t *bytes);
prnu_status prnu_fingerprint_accumulate_persistent(prnu_ctx *ctx, const prnu_camera *cams, int ncams,
                                                   const prnu_params *params, int slots, double wait_budget_ms,
                                                   void *ws, size_t ws_bytes, void *stream);

/* Status of the last persistent launch whose workspace is ws: synchronises
 * `stream`, then returns PRNU_OK, or PRNU_ETIMEOUT when one of its bounded
 * waits gave up; fail_info (nullable, host int[3]) receives the queue item,
 * SDA group and stage of the first wait that gave up. */
prnu_status prnu_persistent_status(prnu_ctx *ctx, const void *ws, size_t ws_bytes, void *stream, int *fail_info);

/* Diagnostic of the bounded waits (no counterpart in the paper): launches
 * the persistent kernel on a one-item queue whose item depends on a count
 * that nothing reaches, so its wait gives up after wait_budget_ms (0 < ms <=
 * 1e4) and prnu_persistent_status then returns PRNU_ETIMEOUT, with the
 * context still usable.  ws: at least 4 KiB. */
prnu_status prnu_persistent_wait_probe(prnu_ctx *ctx, double wait_budget_ms, void *ws, size_t ws_bytes,
                                       void *stream);

/* Fingerprint from the MLE sums, Sec. III-A: K = num/den (division in
 * float64; K = 0 where den == 0), then the optional literature steps named by
 * `flags` (not defined in the paper): PRNU_TO_GRAY, PRNU_ZERO_MEAN,
 * PRNU_WIENER_DFT, applied in that order.
 * num, den: device float32 [C][H][W]; K_out: device float32 [C][H][W], or
 * [1][H][W] with PRNU_TO_GRAY (requires C == 3). */
prnu_status prnu_fingerprint_finalize(prnu_ctx *ctx, const float *num, const float *den, int H, int W, int C,
                                      unsigned flags, const prnu_params *params, float *K_out,
                                      void *ws, size_t ws_bytes, void *stream);

/* Peak-to-correlation energy of a query against a fingerprint (Sec. IV uses
 * PCE with threshold 60; the paper defines it only by citation).  Reading:
 * X = W_q - mean(W_q), Y = K*I_q - mean(K*I_q) (grey planes; C == 3 inputs
 * are converted with the 0.299/0.587/0.114 weights), C(s) = sum_x X(x)
 * Y(x+s) circular (via cuFFT), peak at zero shift,
 *     PCE = sign(C0) C0^2 / mean_{s outside the nbhd x nbhd block around 0} C(s)^2,
 *     NCC = C0 / (|X| |Y|).
 * K: device float32 [H][W] (grey fingerprint); residual_q, img_q: device
 * float32 [C][H][W].  pce_out, ncc_out (nullable), peak_yx (nullable, the
 * (row, col) shift of the maximum of C): host memory, written after this call
 * synchronises `stream`.  nbhd odd, 1 <= nbhd <= min(H, W). */
prnu_status prnu_pce_match(prnu_ctx *ctx, const float *K, const float *residual_q, const float *img_q,
                           int H, int W, int C, int nbhd, double *pce_out, double *ncc_out, int *peak_yx,
                           void *ws, size_t ws_bytes, void *stream);

/* PCE of n queries against one grey fingerprint K (same semantics as n
 * calls of prnu_pce_match, one stream synchronisation): residual_q and img_q
 * are device float32 [n][C][H][W]; pce_out[n], ncc_out[n] (nullable) and
 * peak_yx[2n] (nullable) are host memory. */
prnu_status prnu_pce_match_batch(prnu_ctx *ctx, const float *K, const float *residual_q, const float *img_q, int n,
                                 int H, int W, int C, int nbhd, double *pce_out, double *ncc_out, int *peak_yx,
                                 void *ws, size_t ws_bytes, void *stream);

/* PCE of n (fingerprint, query) pairs, each query against its own grey
 * fingerprint plane: K is device float32 [n][H][W]; otherwise as
 * prnu_pce_match_batch.  Used for block-wise matching (Sec. IV: fingerprints
 * split into disjoint 500 x 500 blocks, each correlated with the same block of
 * the query) and for matrices of fingerprints against queries. */
prnu_status prnu_pce_match_pairs(prnu_ctx *ctx, const float *K, const float *residual_q, const float *img_q, int n,
                                 int H, int W, int C, int nbhd, double *pce_out, double *ncc_out, int *peak_yx,
                                 void *ws, size_t ws_bytes, void *stream);

/* Queries straight from their images: the residual of each query image
 * (the denoiser of prnu_denoise_residual_batch with `params`) matched against
 * K as in prnu_pce_match_batch, without storing the per-channel residuals.
 * Because everything after the shrink is linear, the grey residual of a
 * three-channel query is synthesised once from the 0.299/0.587/0.114
 * combination of the channels' noise coefficients (the same value up to
 * float32 rounding order).  img_q: device float32 [n][C][H][W]; K: device
 * float32 [H][W]; outputs as in prnu_pce_match_batch (host, after a stream
 * synchronisation).  float32 subbands only (EUNSUPPORTED otherwise). */
prnu_status prnu_workspace_size_pce_images(prnu_ctx *ctx, int H, int W, int C, const prnu_params *params, int n,
                                           size_t *bytes);
prnu_status prnu_pce_match_images(prnu_ctx *ctx, const float *K, const float *img_q, int n, int H, int W, int C,
                                  const prnu_params *params, int nbhd, double *pce_out, double *ncc_out,
                                  int *peak_yx, void *ws, size_t ws_bytes, void *stream);

/* prnu_pce_match_images with its outputs left on the device: pce_dev[n],
 * ncc_dev[n] (nullable) and peak_dev[2n] (nullable) are device pointers,
 * written by the last kernel of the call.  Nothing synchronises, so the call
 * can be captured in a CUDA graph after one uncaptured call with the same
 * geometry (which creates any cuFFT plan the geometry needs and sets the
 * correlation kernels' shared-memory attributes).  Errors as
 * prnu_pce_match_images (EINVAL for NULL pointers, n < 1 or a bad nbhd,
 * ENOSPC for a short workspace, EUNSUPPORTED for 16-bit subbands), reported
 * before anything is launched. */
prnu_status prnu_pce_match_images_async(prnu_ctx *ctx, const float *K, const float *img_q, int n, int H, int W,
                                        int C, const prnu_params *params, int nbhd, double *pce_dev, double *ncc_dev,
                                        int *peak_dev, void *ws, size_t ws_bytes, void *stream);

/* prnu_pce_match_images_async in two halves, so that the queries' denoising
 * (which does not involve K) can run on another stream while the fingerprint
 * is extracted.  prnu_pce_images_prepare takes the query images through the
 * wavelet analysis, the shrink and the synthesis down to level 2 and leaves
 * the subbands in ws (size from prnu_workspace_size_pce_images);
 * prnu_pce_images_finish_async, called later (stream-ordered after it) with
 * the same img_q, n, geometry, params and ws, synthesises the grey level-1
 * residual against K and writes the PCE / NCC / peak outputs to the device
 * like prnu_pce_match_images_async.  The results equal those of
 * prnu_pce_match_images.  ws must not be used in between; float32 subbands
 * only (PRNU_EUNSUPPORTED otherwise).  Neither call synchronises. */
prnu_status prnu_pce_images_prepare(prnu_ctx *ctx, const float *img_q, int n, int H, int W, int C,
                                    const prnu_params *params, void *ws, size_t ws_bytes, void *stream);
prnu_status prnu_pce_images_finish_async(prnu_ctx *ctx, const float *K, const float *img_q, int n, int H, int W,
                                         int C, const prnu_params *params, int nbhd, double *pce_dev,
                                         double *ncc_dev, int *peak_dev, void *ws, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * Differentiation.  The chain of Sec. III-A / III-B with the SDA weights made
 * free (the paper's SDA frame is the equal-weight case w_j = 1/d) and sigma0
 * differentiable:
 *   S_i = sum_{j in group i} w_j I_j,   W_i = residual(S_i; sigma0),
 *   K = sum_i W_i S_i / sum_i S_i^2,    PCE of each query against K.
 * Each forward step below has an adjoint ("_backward") that maps the
 * gradient of its outputs to the gradient of its inputs.  The residual's
 * forward keeps every level's detail coefficients (a checkpoint, float32) and
 * its adjoint recomputes the local variances from them.  Requirements: float32
 * subbands (EUNSUPPORTED otherwise) and H, W multiples of 2^levels (no
 * padding; EUNSUPPORTED otherwise).  The derivative is the one of the active
 * branch: away from ties between window means and from min-mean == sigma0^2.
 * All pointers are device pointers unless stated; nothing synchronises.
 * ------------------------------------------------------------------------- */

/* S [g][C][H][W] float32 with S_i = sum_{j in group i} weights[j] * frame_j
 * (uint8 frames as in prnu_sda_average; weights: device float32 [m]). */
prnu_status prnu_sda_weighted(prnu_ctx *ctx, const uint8_t *frames, int m, int H, int W, int C, size_t frame_stride,
                              size_t row_pitch, int d, const float *weights, float *sda_out, void *stream);

/* g_weights[j] = <g_sda[group(j)], frame_j> (written, float32 [m]); the
 * workspace holds at least m * min(H, 64) * 8 bytes (256-byte aligned). */
prnu_status prnu_sda_weighted_backward(prnu_ctx *ctx, const uint8_t *frames, int m, int H, int W, int C,
                                       size_t frame_stride, size_t row_pitch, int d, const float *g_sda,
                                       float *g_weights, void *ws, size_t ws_bytes, void *stream);

/* Workspace of prnu_denoise_residual_ckpt / _backward for n images, and the
 * checkpoint size (bytes of float32 detail coefficients of n images). */
prnu_status prnu_workspace_size_grad(prnu_ctx *ctx, int H, int W, int C, const prnu_params *params, int n,
                                     size_t *ws_bytes, size_t *ckpt_bytes);

/* prnu_denoise_residual_batch that also writes the checkpoint `ckpt`. */
prnu_status prnu_denoise_residual_ckpt(prnu_ctx *ctx, const float *img, int n, int H, int W, int C,
                                       const prnu_params *params, float *residual_out, float *ckpt, void *ws,
                                       size_t ws_bytes, void *stream);

/* Adjoint of the residual: g_img += d<g_residual, W>/d img ([n][C][H][W]),
 * *g_sigma0 += d<g_residual, W>/d sigma0 (device float64, nullable).  ckpt is
 * the forward's checkpoint with the same params. */
prnu_status prnu_denoise_residual_backward(prnu_ctx *ctx, const float *ckpt, int n, int H, int W, int C,
                                           const prnu_params *params, const float *g_residual, float *g_img,
                                           double *g_sigma0, void *ws, size_t ws_bytes, void *stream);

/* MLE fingerprint of n residual/image pairs ([n][C][H][W]), Sec. III-A:
 * num = sum W S, den = sum S^2 ([C][H][W], written), K = num/den (0 where
 * den == 0): [C][H][W], or [H][W] grey (0.299/0.587/0.114) with gray = 1. */
prnu_status prnu_mle_images(prnu_ctx *ctx, const float *residual, const float *img, int n, int H, int W, int C,
                            int gray, float *num, float *den, float *K, void *stream);

/* Adjoint of prnu_mle_images: g_residual, g_img [n][C][H][W] written from
 * g_K (shape of K) and the forward's num, den. */
prnu_status prnu_mle_images_backward(prnu_ctx *ctx, const float *residual, const float *img, int n, int H, int W,
                                     int C, int gray, const float *num, const float *den, const float *g_K,
                                     float *g_residual, float *g_img, void *stream);

prnu_status prnu_workspace_size_pce_backward(prnu_ctx *ctx, int H, int W, int n, size_t *bytes);

/* Adjoint of prnu_pce_match_batch (per_query = 0: one K [H][W]) or of
 * prnu_pce_match_pairs (per_query = 1: K [n][H][W]) with respect to K and the
 * query residuals; g_pce: device float64 [n] (the gradient of each PCE).
 * g_K (written): the shape of K, summed over queries when K is shared;
 * g_residual_q (written): [n][C][H][W].  The queries' images are data. */
prnu_status prnu_pce_backward(prnu_ctx *ctx, const float *K, int per_query, const float *residual_q, const float *img_q,
                              int n, int H, int W, int C, int nbhd, const double *g_pce, float *g_K,
                              float *g_residual_q, void *ws, size_t ws_bytes, void *stream);

/* Autotuner (not part of the paper's method): times every launch shape
 * (strip rows x warps per block) of the level-1 analysis kernel, then every
 * choice of the analysis of levels 2.., the shrink of every level and the
 * synthesis of levels 2.. (prnu_autotune_level), on `images` images of this
 * geometry and storage type, in the workspace (which must hold
 * prnu_workspace_size(..., images) bytes; its contents are overwritten), and
 * keeps the fastest of each in the context for all later calls with that
 * geometry.  Synchronises `stream` (not capturable).  shape_out / ms_out
 * (nullable, host) receive the chosen level-1 shape index and its time per
 * launch. */
prnu_status prnu_autotune(prnu_ctx *ctx, int H, int W, int C, const prnu_params *params, int images, void *ws,
                          size_t ws_bytes, void *stream, int *shape_out, float *ms_out);

/* Pins the level-1 analysis launch shape (index into the tuner's list:
 * 0..5 = 16x4, 32x4, 64x4, 32x2, 32x8, 64x2 strip rows x warps) for this
 * padded geometry and storage type, or with shape = -1 returns it, and every
 * per-level choice of prnu_autotune_level, to the defaults (32x4 and choice
 * 0).  Host only; EINVAL for an index out of range. */
prnu_status prnu_autotune_set(prnu_ctx *ctx, int H, int W, const prnu_params *params, int shape);

/* The tuner's per-level launch choices (prnu_autotune times every choice of
 * kinds 0-2 at every level on its zero planes and keeps the fastest; 0 is the
 * default rule).  kind 0: analysis of level 2..levels (0 tiled 16 x 32 outputs,
 * 1 streaming 16 rows x 4 warps, 2 streaming 32 rows x 2 warps; all give
 * bit-identical results); kind 1: shrink of level 1..levels (0 the register
 * strip where the standard windows and a width that is a multiple of 4 allow
 * it, else the tile; 1 the 32 x 32 tile; the two sum the windows in different
 * orders); kind 2: synthesis of level 2..levels (0 streaming where its grid
 * fills the GPU, else tiled; 1 streaming; 2 tiled); kind 3: the level-1 MLE
 * step of the accumulate calls, level 1 only (0 and 1 the 58 x 32 output tile
 * where it applies -- float32 subbands, even W -- else the 32 x 32 tile; 2 the
 * 32 x 32 tile; both give bit-identical sums).
 * choice >= 0 pins it, -1 returns it to the default, -2 only reads it;
 * *current (nullable) receives the choice in force.  Host only. */
prnu_status prnu_autotune_level(prnu_ctx *ctx, int H, int W, const prnu_params *params, int kind, int level,
                                int choice, int *current);

/* Index checks (not part of the paper's method).  The debug build of the
 * library (libprnu_debug.so, compiled with PRNU_DEBUG; same entry points)
 * checks the global-memory indices of its kernels against the extents their
 * arguments imply; the first failed check of each source file records the
 * line and the index and the access is skipped (no trap).  This call
 * synchronises the context's device, then returns PRNU_OK when no check has
 * failed since the previous call, or PRNU_EDEBUG with "file:line index" of the
 * first failure in *where (host buffer of where_len bytes, nullable); the
 * records are cleared.  The release build returns PRNU_EUNSUPPORTED. */
prnu_status prnu_debug_status(prnu_ctx *ctx, char *where, size_t where_len);

/* Per-kernel profiling (not part of the paper's method).  Every kernel launch
 * is counted per kernel name.  With profiling on, each launch (and each cuFFT
 * call, named cufft_*) is also bracketed by CUDA events recorded on its
 * stream; the events are drawn from a pool the context owns.  Under stream
 * capture the events become event-record nodes of the graph (launches are
 * counted once, at capture), so prnu_profile_read then reports the device time
 * of the graph's latest replay.  Destroy such a graph before
 * prnu_profile_reset, which returns its events to the pool. */
prnu_status prnu_profile_enable(prnu_ctx *ctx, int on);

/* Restricts the event timing of prnu_profile_enable to the kernels named in
 * `names`, a comma-separated list of profile names ("shrink,sda_sum"); the
 * other launches are still counted.  NULL or "" times every launch again.
 * Host only; the string is copied. */
prnu_status prnu_profile_select(prnu_ctx *ctx, const char *names);

/* Clear the counters and recorded events (waits for the recorded events). */
prnu_status prnu_profile_reset(prnu_ctx *ctx);

/* Kernel number `index` (0-based, in order of first launch): its name
 * (NUL-terminated, truncated to name_len), launches since the last reset, the
 * summed device time in ms of its launches recorded while profiling was on
 * (waits for those events) and the algorithmic bytes of the counted launches
 * (each input byte read once, each output byte written once; 0 for cuFFT).
 * Any output pointer may be NULL.  PRNU_EINVAL past the last kernel. */
prnu_status prnu_profile_read(prnu_ctx *ctx, int index, char *name, size_t name_len, long long *launches,
                              double *total_ms, double *bytes);

#ifdef __cplusplus
}
#endif

#endif /* PRNU_H */
