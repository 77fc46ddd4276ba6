// kernels.cuh -- argument blocks and launchers of the libprnu kernels.
#pragma once

#include <cufft.h>

#include "common.cuh"

namespace prnu {

// k_sda.cu
struct SdaArgs {
    const uint8_t *frames;  // uint8 frames, or fp16 frames when frame_half (byte pointer)
    int frame_half;
    long long frame_stride, row_pitch;
    int m, H, W, C, d;
    int g0, G;      // groups g0 .. g0+G-1 are produced, output index g - g0
    float *out;     // [G][C][H][W]
    int mean;       // 1: write sum/count (correctly rounded), 0: the exact sum
    const GroupDesc *gd;  // multi-camera pass: per-group frames/strides/count (frames..d, g0 unused)
    int blocks_per_sm;    // grid cap (0: fill the SMs); frames read over the host link need few blocks
};
cudaError_t launch_put_desc(const PassDesc &pd, PassDesc *dst, cudaStream_t st);
cudaError_t launch_sda(const SdaArgs &a, int num_sms, cudaStream_t st);

// k_dwt.cu
struct AnaArgs {
    const float *inh;   // level 1: planes [P][H][W] virtually mirror-padded to R x Cc
    const float *inl;   // levels >= 2: low parts [P][R][Cc]; level 1: unused
    int R, Cc;          // input dims at this level (even)
    int H, W;           // level 1: unpadded source dims
    int P;
    float *LLh, *LLl;   // [P][R/2][Cc/2]; null on the last level
    void *LH, *HL, *HH;  // detail subbands, storage type sdt
    int sdt;
    PlaneScale sc;
    int scale_on;
    Filt f;
};
// level-1 launch shapes (strip rows x warps per block) of the autotuner
constexpr int kStreamShapes = 6;
constexpr int kStreamShapeDefault = 1;  // 32 rows x 4 warps
constexpr int kStreamShapeDims[kStreamShapes][2] = {{16, 4}, {32, 4}, {64, 4}, {32, 2}, {32, 8}, {64, 2}};
cudaError_t launch_analysis(const AnaArgs &a, bool level1, cudaStream_t st, int shape = kStreamShapeDefault);

// k_sda_dwt.cu: the group sums of s (into s.out, exact sums) and the level-1
// analysis of a (a.inh unused) in one kernel, where sda_dwt_applies: uint8
// frames, C = 1 or 3, padded width == W, W*C a multiple of 16, 16-byte
// aligned frames and strides, groups of 1..257 frames.  A multi-camera pass
// (s.gd set) passes the host copy of its descriptor as pd (nullptr
// otherwise).  strips: output-row strips per column (0: about two blocks per
// SM).
bool sda_dwt_applies(const SdaArgs &s, const AnaArgs &a, const PassDesc *pd);
cudaError_t launch_sda_dwt(const SdaArgs &s, const AnaArgs &a, const PassDesc *pd, int num_sms, cudaStream_t st,
                           int strips = 0);
// tuner choices of the other launches (0 = the default rule)
// levels >= 2 analysis: 0 tiled 16 x 32, 1 streaming 16 rows x 4 warps, 2 streaming 32 x 2
constexpr int kAnaChoices = 3;
// shrink: 0 strip where it applies (standard windows, width % 4 == 0), else tiled; 1 tiled
constexpr int kShrinkChoices = 2;
// synthesis (levels >= 2): 0 streaming where its grid fills the GPU, else tiled; 1 streaming; 2 tiled
constexpr int kSynChoices = 3;
// level-1 MLE step: 0 and 1 the 58 x 32 wide tile where it applies (float32 subbands, even W), else
// the 32 x 32 tile; 2 the 32 x 32 tile
constexpr int kFinalChoices = 3;
enum TuneKind : int { kTuneAnalysis = 0, kTuneShrink = 1, kTuneSynthesis = 2, kTuneFinal = 3 };

// k_shrink.cu
struct ShrinkArgs {
    const void *in;       // [nplanes][R][Cc], storage type sdt
    void *out;            // [nplanes][R][Cc] (must not alias `in`)
    int sdt;
    int R, Cc, nplanes;
    float s2;             // sigma0^2, or taken from s2_dev[1] when s2_dev != null
    const double *s2_dev;
    Win win;
};
cudaError_t launch_shrink(const ShrinkArgs &a, cudaStream_t st, int choice = 0);

// k_idwt.cu
struct SynArgs {
    const void *LL;    // noise LL at this level [P][Rc][Cc], or null (zero); storage type sdt
    const void *LH, *HL, *HH;
    int Rc, Cc, P;     // coefficient dims; output is 2Rc x 2Cc
    void *out;         // [P][2Rc][2Cc]
    int sdt;
    int gray3;         // float32 only: output plane z synthesises 0.299/0.587/0.114 of detail
                       // planes 3z, 3z+1, 3z+2 (LL is already grey: plane z)
    Filt f;
};
struct FinalArgs {
    const void *LL;    // level-1 noise LL [P][Rc][Cc], or null (one-level transform); storage type sdt
    const void *LH, *HL, *HH;
    int sdt;
    int compensated;   // MLE mode: num, den are [2][C][H][W] float-float pairs (hi, then lo)
    int Rc, Cc;        // Hp/2, Wp/2
    int H, W, C, G;    // crop and plane map: image i, channel c -> plane i*C + c
    const float *X;    // MLE mode: group sums [G][C][H][W]
    PlaneScale sc;
    float *res_out;    // residual mode: [G*C][H][W]
    int accumulate;    // residual mode: res_out += W instead of res_out = W
    float *num, *den;  // MLE mode: [C][H][W]
    const GroupDesc *gd;    // multi-camera MLE: group -> camera (groups of a camera are consecutive)
    const CamDesc *cams;    // multi-camera MLE: per-camera num/den
    // PCE mode (float32 subbands): per query z, X = grey W (the grey synthesis
    // of the detail planes, as in gray3), Y = K grey(I); block partial sums of
    // X, X^2, Y, Y^2 (float64) at part_m[z][block][4]
    int pce;
    const float *Kq;        // [H][W], or one per query at stride k_stride
    long long k_stride;
    const float *Iq;        // query images [G][C][H][W]
    float *Xo, *Yo;         // [G][H][W]
    double *part_m;
    Filt f;
};
// blocks per query of the PCE-mode level-1 kernel (its partial-sum count)
int final_pce_blocks(int Rc, int Cc);
cudaError_t launch_synthesis(const SynArgs &a, cudaStream_t st, int choice = 0);
cudaError_t launch_final(const FinalArgs &a, bool mle, cudaStream_t st, int choice = 0);

// k_fft.cu
cudaError_t launch_divide(const float *num, const float *den, const float *num_lo, const float *den_lo, long long hw,
                          int C, int gray, float *K, int sms, cudaStream_t st);
cudaError_t launch_zero_mean(float *K, int H, int W, double *colmean, double *rowmean, double *part, int sms,
                             cudaStream_t st);
cudaError_t launch_mean_var(const float *v, long long n, double *part, int nb, double *tmp, double *out,
                            cudaStream_t st, bool zero_mean = false);
cudaError_t launch_magnitude_half(const cufftComplex *Fh, int H, int W, float inv_sqrt_n, float *M, int sms,
                                  cudaStream_t st);
cudaError_t launch_apply_ratio_half(cufftComplex *Fh, const float *M, const float *Mn, int H, int W, float scale,
                                    int sms, cudaStream_t st);
cudaError_t launch_pce_prep(const float *K, long long k_stride, const float *Wq, const float *Iq, long long hw, int C,
                            int n, int nb, float *X, float *Y, double *part, cudaStream_t st);
cudaError_t launch_cross_spectrum(const cufftComplex *FX, const cufftComplex *FY, long long nh, int n,
                                  cufftComplex *Z, int sms, cudaStream_t st);
cudaError_t launch_pce_reduce(const float *Cr, int H, int W, int r, int n, int nb, double *part_e, float *part_v,
                              long long *part_i, const double *part_m, int nbm, void *out, cudaStream_t st);
// per-query PCE scalars written by the reduction (device)
struct PceScalars {
    double c0, energy;
    long long peak_idx;
    double sx, sxx, sy, syy;
};
size_t pce_scalars_bytes();
cudaError_t launch_pce_final(const float *c0, long long c0_stride, int n, const double *part_e, const float *part_v,
                             const long long *part_i, int nb, const double *part_m, int nbm, void *out,
                             cudaStream_t st);

// k_corr.cu -- PCE correlation by our own mixed-radix FFTs
constexpr int kMaxFftPasses = 16;
struct FftSteps {
    int L = 0, np = 0;
    unsigned long long radix = 0;  // radix of pass i (8, 4, 2, 3, 5 or 7) in bits 4i..4i+3
    __host__ __device__ int r(int i) const { return (int)((radix >> (4 * i)) & 15u); }
};
bool fft_steps(int L, FftSteps *p);
// true when W is even and W/2 and H factor into 2, 3, 5, 7 within the
// shared-memory limits of the kernels
bool corr_fft_supported(int H, int W);
size_t corr_twiddle_count(int H, int W);  // float2 entries
int corr_pitch(int W);                    // complex bins per half-spectrum row (W/2 + 1, padded to 4)
int corr_rows_blocks(int H, int W, int nb);
// stage 0: twiddles + row FFTs of the 2n planes XY into F; 1: column FFTs,
// cross spectrum and inverse column FFTs (in place over the X half of F);
// 2: inverse row FFTs and the PCE partials (corr_rows_blocks per query).
cudaError_t launch_corr_fft(const float *XY, float2 *F, float2 *tw, int n, int H, int W, int r, int nb,
                            double *part_e, float *part_v, long long *part_i, float *c0, int sms, cudaStream_t st,
                            int stage);
cudaError_t launch_pce_outputs(const void *sc, int n, long long hw, int W, int nbhd, double *pce, double *ncc,
                               int *peak, cudaStream_t st);

// k_grad.cu -- adjoints
struct ShrinkBwdArgs {
    const float *c;    // forward detail coefficients (checkpoint) [nplanes][R][Cc]
    const float *gn;   // gradient of the noise coefficients
    float *gc;         // gradient of the coefficients (written)
    int R, Cc, nplanes;
    float s2, two_sigma0;
    Win win;
    double *g_sigma;   // += dL/dsigma0 (nullable)
};
cudaError_t launch_sda_weighted(const SdaArgs &a, const float *wts, int num_sms, cudaStream_t st);
int sda_wgrad_blocks(int H);
cudaError_t launch_sda_wgrad(const SdaArgs &a, const float *gS, double *part, float *gw, cudaStream_t st);
cudaError_t launch_mle_images(const float *res, const float *img, int n, int C, long long hw, int gray, float *num,
                              float *den, float *K, int sms, cudaStream_t st);
cudaError_t launch_mle_images_bwd(const float *res, const float *img, int n, int C, long long hw, int gray,
                                  const float *num, const float *den, const float *gK, float *gres, float *gimg,
                                  int sms, cudaStream_t st);
cudaError_t launch_shrink_bwd(const ShrinkBwdArgs &a, cudaStream_t st);
cudaError_t launch_pce_gfield(float *Cr, int H, int W, int r, int n, const void *scal, const double *g,
                              cudaStream_t st);
cudaError_t launch_pce_spectra_bwd(cufftComplex *FX, cufftComplex *FY, const cufftComplex *FG, long long nh, int n,
                                   int sms, cudaStream_t st);
cudaError_t launch_pce_bwd_out(const float *gYraw, const float *gXraw, const float *Iq, int n, int C, long long hw,
                               float inv_n, int per_query, float *gK, float *gres, int sms, cudaStream_t st);
void pce_unpack(const void *p, int q, double *c0, double *energy, long long *peak_idx, double *sx, double *sxx,
                double *sy, double *syy);

// k_persist.cu -- the multi-camera pipeline as one persistent launch over a
// device work queue of (group, stage, tile) items.
// Stages of a group with L levels: 0 SDA sums; l = 1..L analysis of level l;
// L + l shrink of level l; 3L + 1 - l synthesis of level l (l = L..2); 3L the
// level-1 synthesis with the MLE sums.
constexpr int kPMaxStages = 3 * kMaxLevels + 1;
constexpr int kPMaxGeos = 8;
constexpr int kPProbeStage = kPMaxStages;  // a diagnostic item that waits on a count nothing reaches
// tiles per queue item (more work per claim, wait and count): SDA sums,
// analysis, shrink, synthesis, level-1 synthesis + MLE
constexpr int kPTilesSda = 1, kPTilesAna = 4, kPTilesShr = 4, kPTilesSyn = 4, kPTilesFin = 2;
struct PGroup {
    const uint8_t *frames;
    long long frame_stride, row_pitch;
    int n;     // frames in the group
    int cam;   // index into the camera table
    int geo;   // index into the geometry table
    int prev;  // the camera's previous group in this launch (its MLE sums come first), or -1
};
struct PCam {
    float *num, *den;
};
struct PGeo {
    int H, W, C, Hp, Wp;
    int cnt[kPMaxStages];  // work items per stage
    // byte offsets within a slot (the single-plane-group layout of the pipeline)
    long long X, LLh[kMaxLevels + 1], LLl[kMaxLevels + 1], Rn[kMaxLevels + 1], D[kMaxLevels + 1],
        N[kMaxLevels + 1];
};
// a run of consecutive queue items of one stage of one group: queue items
// start .. next segment's start - 1 are that stage's items first, first + 1, ...
struct PSeg {
    int start, group, stage, first;
};
struct PHeader {
    int next;    // queue head (claimed items)
    int status;  // PRNU_OK, or PRNU_ETIMEOUT once a wait gave up
    int fail_item, fail_group, fail_stage, fail_blocks;
    int pad[2];
};
struct PArgs {
    PHeader *hdr;
    const PGroup *groups;
    const PCam *cams;
    const PGeo *geos;
    const PSeg *segs;
    int *done;  // [G][NS] completed items per (group, stage)
    char *slots;
    long long slot_bytes;
    int nslots, L, NS, nseg, total, G;
    float s2;
    Win win;
    Filt f;
    long long budget_ns;  // longest wait on one dependency
};
// template switches: compensated MLE sums, the standard 3/5/7/9 windows
cudaError_t launch_persist(const PArgs &a, bool comp, bool std_win, int blocks, cudaStream_t st);
int persist_blocks_per_sm(bool comp, bool std_win);
constexpr int kPutChunk = 24576;  // bytes per by-value copy launch
cudaError_t launch_put_bytes(const void *src, size_t n, void *dst, cudaStream_t st);

}  // namespace prnu
