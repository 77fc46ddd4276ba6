"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: SDA mean bit-exact (both sides round the exact mean once);
residual max-abs <= 1e-3 in 0..255 units; fingerprint relative L2 <= 1e-5;
PCE within 0.1 %.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1909_04573_gb300 import prnu as P
from paper_1909_04573_gb300 import synth

pytestmark = pytest.mark.gpu

RES_TOL = 1e-3
K_TOL = 1e-5
PCE_TOL = 1e-3


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_04573_gb300 import build
    build.build()
    c = P.Context(0)
    yield c
    c.close()


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _frames(H, W, C, m, seed=0, drift=0.0):
    return synth.frames(synth.Camera(H=H, W=W, C=C, camera_id=seed), m, drift_px=drift).numpy()


# ------------------------------------------------------------------- SDA ----
@pytest.mark.parametrize("H,W,C,m,d", [(16, 16, 1, 5, 2), (37, 50, 3, 11, 4), (64, 80, 3, 20, 20),
                                       (33, 21, 1, 7, 1), (256, 256, 1, 64, 8)])
def test_sda_average_bit_exact(ctx, H, W, C, m, d):
    fr = np.random.default_rng(H * W + m).integers(0, 256, size=(m, H, W, C), dtype=np.uint8)
    got = ctx.sda_average(_dev(fr), d).cpu().numpy()
    ref = O.sda_average(fr, d).astype(np.float32)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("H,W,C,m,d", [(64, 80, 3, 600, 300), (40, 52, 3, 70, 9), (96, 100, 3, 40, 40), (17, 35, 3, 30, 7),
                                       (1080, 1920, 3, 12, 5)])
def test_sda_long_groups_and_segment_tails(ctx, H, W, C, m, d):
    """Row segments that end mid-chunk, groups longer than 256 frames (the
    16-bit lanes are flushed), ragged last groups, L2 prefetches that reach
    the last frame; exact sums (as means, bit for bit)."""
    fr = np.random.default_rng(H * W * C + m).integers(0, 256, size=(m, H, W, C), dtype=np.uint8)
    got = ctx.sda_average(_dev(fr), d).cpu().numpy()
    ref = O.sda_average(fr, d).astype(np.float32)
    np.testing.assert_array_equal(got, ref)


def test_sda_average_strided_frames(ctx):
    rng = np.random.default_rng(5)
    big = rng.integers(0, 256, size=(9, 40, 70, 3), dtype=np.uint8)
    view = _dev(big)[:, 2:34, 3:51, :]          # row pitch 210 B, frame stride 8400 B
    got = ctx.sda_average(view, 3).cpu().numpy()
    ref = O.sda_average(np.ascontiguousarray(big[:, 2:34, 3:51, :]), 3).astype(np.float32)
    np.testing.assert_array_equal(got, ref)


# -------------------------------------------------------------- residual ----
@pytest.mark.parametrize("H,W,C", [(16, 16, 1), (37, 50, 1), (64, 64, 3), (100, 300, 1), (256, 256, 1),
                                   (272, 480, 3)])
def test_denoise_residual_matches_oracle(ctx, H, W, C):
    fr = _frames(H, W, C, 1, seed=H + W)
    img = fr[0].transpose(2, 0, 1).astype(np.float32)
    got = ctx.denoise_residual(_dev(img)).cpu().numpy()
    ref = O.residual(img.astype(np.float64))
    assert np.abs(got - ref).max() <= RES_TOL
    assert _rel(got, ref) <= 1e-5


@pytest.mark.parametrize("levels,sigma0,windows", [(1, 3.0, (3, 5, 7, 9)), (2, 2.0, (3,)), (5, 3.0, (5, 9)),
                                                   (4, 0.5, (1, 3)), (3, 6.0, (9, 7, 5, 3))])
def test_denoise_residual_parameters(ctx, levels, sigma0, windows):
    img = _frames(64, 96, 1, 1, seed=11)[0].transpose(2, 0, 1).astype(np.float32)
    got = ctx.denoise_residual(_dev(img), P.default_params(levels, sigma0, windows)).cpu().numpy()
    ref = O.residual(img.astype(np.float64), O.Params(levels=levels, sigma0=sigma0, windows=tuple(windows)))
    assert np.abs(got - ref).max() <= RES_TOL


def test_denoise_residual_degenerate_cases(ctx):
    const = np.full((1, 48, 48), 131.0, np.float32)
    assert np.abs(ctx.denoise_residual(_dev(const)).cpu().numpy()).max() <= 1e-4
    img = _frames(48, 48, 1, 1, seed=2)[0].transpose(2, 0, 1).astype(np.float32)
    w0 = ctx.denoise_residual(_dev(img), P.default_params(sigma0=0.0)).cpu().numpy()
    assert np.all(w0 == 0.0)


# ------------------------------------------------------------ fingerprint ---
def _accumulate(ctx, fr, d, images_per_pass=None):
    m, H, W, C = fr.shape
    num = torch.zeros((C, H, W), dtype=torch.float32, device="cuda")
    den = torch.zeros_like(num)
    ctx.fingerprint_accumulate(_dev(fr), d, num, den, images_per_pass=images_per_pass)
    return num.cpu().numpy(), den.cpu().numpy()


@pytest.mark.parametrize("H,W,C,m,d,drift", [(256, 256, 1, 64, 8, 0.0),    # small config: 8 SDA groups
                                              (64, 80, 1, 37, 8, 0.0),      # ragged last group
                                              (48, 64, 1, 12, 1, 0.0),      # per-frame estimator
                                              (96, 128, 3, 30, 10, 2.0)])   # RGB, drifting scene
def test_fingerprint_accumulate_matches_oracle(ctx, H, W, C, m, d, drift):
    fr = _frames(H, W, C, m, seed=m, drift=drift)
    num, den = _accumulate(ctx, fr, d)
    onum, oden = O.fingerprint_accumulate(fr, d)
    assert _rel(den, oden) <= 1e-6
    assert _rel(num, onum) <= K_TOL
    K = ctx.fingerprint_finalize(_dev(num), _dev(den)).cpu().numpy()
    assert _rel(K, O.fingerprint_finalize(onum, oden)) <= K_TOL


def test_multipass_accumulate_and_determinism(ctx):
    fr = _frames(64, 64, 3, 24, seed=4)
    n1, d1 = _accumulate(ctx, fr, 4)                      # all six groups in one pass
    n2, d2 = _accumulate(ctx, fr, 4, images_per_pass=1)   # a smaller workspace: several passes
    n3, d3 = _accumulate(ctx, fr, 4)
    np.testing.assert_array_equal(n1, n3)                 # run to run
    np.testing.assert_array_equal(d1, d3)
    assert _rel(n2, n1) <= 1e-6 and _rel(d2, d1) <= 1e-6


@pytest.mark.parametrize("passes", [2, 3, 8])
def test_pipelined_accumulate_equals_one_stream_and_replays(ctx, passes):
    """prnu_params.pipeline_passes: the group sums of the next pass on the
    context's side stream beside the current pass's denoising (two pass
    layouts, events); eager and captured in a CUDA graph, it gives the sums of
    the one-stream call."""
    fr = torch.as_tensor(_frames(64, 96, 3, 37, seed=8)).cuda()
    C, H, W = 3, 64, 96
    ref_n, ref_d = torch.zeros((C, H, W), device="cuda"), torch.zeros((C, H, W), device="cuda")
    ctx.fingerprint_accumulate(fr, 4, ref_n, ref_d)
    prm = P.default_params(pipeline_passes=passes)
    num, den = torch.zeros_like(ref_n), torch.zeros_like(ref_d)
    ctx.fingerprint_accumulate(fr, 4, num, den, params=prm)
    torch.cuda.synchronize()
    # the passes add their groups' sums into num/den one pass at a time (the
    # one-stream call has a single pass here): equal to float32 rounding
    assert _rel(num.cpu().numpy(), ref_n.cpu().numpy()) <= 1e-6
    assert _rel(den.cpu().numpy(), ref_d.cpu().numpy()) <= 1e-6
    eager_n, eager_d = num.clone(), den.clone()
    f, m, Hh, Ww, Cc, fs, rp = ctx._frames_geometry(fr)
    nb = P.prnu_workspace_size(ctx.ctx, H, W, C, prm, 10)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            num.zero_()
            den.zero_()
            P.prnu_fingerprint_accumulate(ctx.ctx, f.data_ptr(), m, H, W, C, fs, rp, 4, prm, num.data_ptr(),
                                          den.data_ptr(), ws.data_ptr(), nb, side.cuda_stream)
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(2):
        num.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(num, eager_n) and torch.equal(den, eager_d)


@pytest.mark.parametrize("pinned", [True, False])
def test_accumulate_host_equals_device(ctx, pinned):
    """Page-locked frames are read in place (zero copy), pageable ones are
    staged through the workspace; both equal the device path."""
    fr = _frames(48, 64, 3, 20, seed=6)
    num = torch.zeros((3, 48, 64), dtype=torch.float32, device="cuda")
    den = torch.zeros_like(num)
    host = torch.from_numpy(fr).pin_memory() if pinned else torch.from_numpy(fr.copy())
    ctx.fingerprint_accumulate_host(host, 5, num, den, groups_per_pass=2)
    n2, d2 = _accumulate(ctx, fr, 5, images_per_pass=2)
    torch.cuda.synchronize()
    assert _rel(num.cpu().numpy(), n2) <= 1e-6
    assert _rel(den.cpu().numpy(), d2) <= 1e-6


@pytest.mark.parametrize("flags", [0, P.PRNU_ZERO_MEAN, P.PRNU_TO_GRAY, P.PRNU_TO_GRAY | P.PRNU_ZERO_MEAN,
                                   P.PRNU_WIENER_DFT, P.PRNU_TO_GRAY | P.PRNU_ZERO_MEAN | P.PRNU_WIENER_DFT])
def test_finalize_flags(ctx, flags):
    rng = np.random.default_rng(flags)
    C, H, W = 3, 60, 84
    den = rng.uniform(1e4, 5e4, size=(C, H, W)).astype(np.float32)
    num = (den * rng.normal(0, 0.01, size=(C, H, W))).astype(np.float32)
    den[0, 3, 5] = 0.0
    got = ctx.fingerprint_finalize(_dev(num), _dev(den), flags).cpu().numpy()
    ref = O.fingerprint_finalize(num.astype(np.float64), den.astype(np.float64), flags)
    assert got.shape == ref.shape
    assert _rel(got, ref) <= K_TOL


# ------------------------------------------------------------------- PCE ----
# own-FFT geometries (radix 8/4/2/3/5/7 factors, column tiles with a ragged
# tail, two-row blocks for W/2 > 1024) and cuFFT ones (prime factors)
@pytest.mark.parametrize("H,W,C", [(64, 64, 1), (96, 80, 3), (256, 256, 1), (84, 140, 1), (50, 2240, 1),
                                   (74, 94, 1), (1080, 1920, 1)])
def test_pce_matches_oracle(ctx, H, W, C):
    rng = np.random.default_rng(H * C)
    K = rng.normal(0, 0.01, size=(H, W))
    Iq = rng.uniform(40, 220, size=(C, H, W))
    Wq = K[None] * Iq + rng.normal(0, 0.7, size=(C, H, W))
    pce, ncc, peak = ctx.pce_match(_dev(K.astype(np.float32)), _dev(Wq.astype(np.float32)),
                                   _dev(Iq.astype(np.float32)))
    r = O.pce_match(K, O.to_gray(Wq.astype(np.float32)), O.to_gray(Iq.astype(np.float32)))
    assert abs(pce - r.pce) <= PCE_TOL * abs(r.pce)
    assert abs(ncc - r.ncc) <= 1e-4 * abs(r.ncc)
    assert peak == r.peak == (0, 0)


def test_pce_images_prepare_then_finish_overlapping_an_extraction(ctx):
    """The query half split in two (prepare on a side stream in its own
    context while the fingerprint is accumulated, finish after the join)
    gives the PCE / NCC / peak of prnu_pce_match_images."""
    H, W, C, n = 200, 320, 3, 3
    cam = synth.Camera(H=H, W=W, C=C, camera_id=91)
    fr = synth.frames(cam, 24, device="cuda")
    qf = torch.cat([synth.frames(cam, n - 1, stream=1, device="cuda"),
                    synth.frames(synth.foreign(cam), 1, stream=1, device="cuda")])
    q = ctx.sda_average(qf, 1)
    flags = P.PRNU_TO_GRAY | P.PRNU_ZERO_MEAN | P.PRNU_WIENER_DFT
    num = torch.zeros((C, H, W), device="cuda")
    den = torch.zeros_like(num)
    qctx = P.Context(0)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        qctx.pce_images_prepare(q)
    ctx.fingerprint_accumulate(fr, 8, num, den)
    K = ctx.fingerprint_finalize(num, den, flags)
    torch.cuda.current_stream().wait_stream(side)
    out = qctx.pce_images_finish_async(K[0], q)
    ref = ctx.pce_match_images(K[0], q)
    torch.cuda.synchronize()
    for i, (p, c, k) in enumerate(ref):
        assert out[0][i].item() == p and out[1][i].item() == c
        assert tuple(out[2][i].tolist()) == tuple(k)
    assert ref[0][0] > 60 and abs(ref[-1][0]) < 60
    qctx.close()


@pytest.mark.parametrize("H,W,dy,dx", [(84, 140, 5, -9), (96, 80, -30, 17), (74, 94, 3, 40)])
def test_pce_peak_follows_a_circular_shift(ctx, H, W, dy, dx):
    """The query's noise is the fingerprint pattern shifted circularly by
    (dy, dx): the correlation peak moves to that shift (bit-exact index
    against the oracle) and the PCE at zero shift collapses."""
    rng = np.random.default_rng(H + W)
    K = rng.normal(0, 0.01, size=(H, W))
    Iq = rng.uniform(40, 220, size=(1, H, W))
    Wq = np.roll(K[None] * Iq, (-dy, -dx), axis=(1, 2)) + rng.normal(0, 0.3, size=(1, H, W))
    pce, ncc, peak = ctx.pce_match(_dev(K.astype(np.float32)), _dev(Wq.astype(np.float32)),
                                   _dev(Iq.astype(np.float32)))
    r = O.pce_match(K, O.to_gray(Wq.astype(np.float32)), O.to_gray(Iq.astype(np.float32)))
    assert peak == r.peak == (dy % H, dx % W)
    assert abs(pce - r.pce) <= PCE_TOL * max(abs(r.pce), 1.0)
    assert abs(pce) < 60


def test_planted_camera_end_to_end(ctx):
    # 64 grayscale 256x256 frames, SDA groups of 8; one same-camera and one
    # foreign query; PCE threshold 60 (Sec. IV) separates them on both sides
    cam = synth.Camera(H=256, W=256, C=1, camera_id=21)
    fr = synth.frames(cam, 64).numpy()
    num, den = _accumulate(ctx, fr, 8)
    K = ctx.fingerprint_finalize(_dev(num), _dev(den))
    onum, oden = O.fingerprint_accumulate(fr, 8)
    oK = O.fingerprint_finalize(onum, oden)[0]
    for qcam, positive in ((cam, True), (synth.foreign(cam), False)):
        q = synth.frames(qcam, 1, stream=1).numpy()[0].transpose(2, 0, 1).astype(np.float32)
        wq = ctx.denoise_residual(_dev(q))
        pce, _, _ = ctx.pce_match(K[0], wq, _dev(q))
        ref = O.pce_match(oK, O.residual(q.astype(np.float64))[0], q[0].astype(np.float64)).pce
        assert abs(pce - ref) <= PCE_TOL * abs(ref)
        assert (pce > 60) == positive


# ------------------------------------------------------------ full size -----
@pytest.mark.slow
def test_full_hd_rgb_sda50_two_groups(ctx):
    # 1920x1080 RGB with a drifting scene, SDA groups of 50 (the video-scale
    # geometry: 1080 rows need mirror padding to 1088); two groups
    cam = synth.Camera(H=1080, W=1920, C=3, camera_id=31)
    fr = synth.frames(cam, 100, device="cuda", drift_px=2.0)
    num = torch.zeros((3, 1080, 1920), dtype=torch.float32, device="cuda")
    den = torch.zeros_like(num)
    ctx.fingerprint_accumulate(fr, 50, num, den)
    onum, oden = O.fingerprint_accumulate(fr.cpu().numpy(), 50)
    assert _rel(den.cpu().numpy(), oden) <= 1e-6
    assert _rel(num.cpu().numpy(), onum) <= K_TOL
    # one SDA frame's residual, all three channels
    sda = ctx.sda_average(fr[:50], 50)[0]
    got = ctx.denoise_residual(sda).cpu().numpy()
    ref = O.residual(O.sda_average(fr[:50].cpu().numpy(), 50)[0])
    assert np.abs(got - ref).max() <= RES_TOL


# --------------------------------------------------------------- errors -----
def test_invalid_arguments_are_rejected(ctx):
    img = torch.zeros((1, 8, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(P.PrnuError) as e:
        ctx.denoise_residual(img)
    assert e.value.status == P.PRNU_EINVAL
    fr = torch.zeros((4, 32, 32, 2), dtype=torch.uint8, device="cuda")
    with pytest.raises(P.PrnuError):
        ctx.sda_average(fr, 2)
    with pytest.raises(P.PrnuError):
        ctx.denoise_residual(torch.zeros((1, 32, 32), device="cuda"), P.default_params(windows=(4,)))
    p = P.default_params()
    n = P.prnu_workspace_size(ctx.ctx, 64, 64, 1, p, 1)
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    x = torch.zeros((1, 64, 64), device="cuda")
    with pytest.raises(P.PrnuError) as e:
        P.prnu_denoise_residual(ctx.ctx, x.data_ptr(), 64, 64, 1, p, torch.empty_like(x).data_ptr(),
                                ws.data_ptr(), 1024, ctx._stream())
    assert e.value.status == P.PRNU_ENOSPC


def test_empty_inputs_and_out_of_range_group_sizes_are_rejected(ctx):
    """No frames, no queries, and SDA group sizes outside [1, m] (Sec. III-B
    groups d consecutive frames of the m given) are rejected with EINVAL
    before anything is launched: num / den keep their contents."""
    H, W, C = 32, 64, 3
    fr = synth.frames(synth.Camera(H=H, W=W, C=C, camera_id=5), 4).cuda()
    p = P.default_params()
    n = P.prnu_workspace_size(ctx.ctx, H, W, C, p, 4)
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    num = torch.full((C, H, W), 7.0, device="cuda")
    den = torch.full_like(num, 3.0)
    fs, rp = H * W * C, W * C
    for m, d in ((0, 1), (0, 0), (4, 0), (4, 5)):
        with pytest.raises(P.PrnuError) as e:
            P.prnu_fingerprint_accumulate(ctx.ctx, fr.data_ptr(), m, H, W, C, fs, rp, d, p, num.data_ptr(),
                                          den.data_ptr(), ws.data_ptr(), n, ctx._stream())
        assert e.value.status == P.PRNU_EINVAL, (m, d)
    out = torch.zeros((1, C, H, W), device="cuda")
    with pytest.raises(P.PrnuError) as e:
        P.prnu_sda_average(ctx.ctx, fr.data_ptr(), 0, H, W, C, fs, rp, 1, out.data_ptr(), ctx._stream())
    assert e.value.status == P.PRNU_EINVAL
    K = torch.zeros((H, W), device="cuda")
    q = torch.zeros((1, C, H, W), device="cuda")
    nq = P.prnu_workspace_size_pce_images(ctx.ctx, H, W, C, p, 1)
    wq = torch.empty(nq, dtype=torch.uint8, device="cuda")
    with pytest.raises(P.PrnuError) as e:
        P.prnu_pce_match_images(ctx.ctx, K.data_ptr(), q.data_ptr(), 0, H, W, C, p, 11, wq.data_ptr(), nq,
                                ctx._stream())
    assert e.value.status == P.PRNU_EINVAL
    torch.cuda.synchronize()
    assert bool((num == 7.0).all()) and bool((den == 3.0).all())


# --------------------------------------------------------------- batches ----
def test_denoise_residual_batch_matches_oracle(ctx):
    imgs = np.stack([_frames(72, 104, 3, 1, seed=40 + i)[0].transpose(2, 0, 1) for i in range(5)]).astype(np.float32)
    got = ctx.denoise_residual_batch(_dev(imgs)).cpu().numpy()
    for i in range(5):
        ref = O.residual(imgs[i].astype(np.float64))
        assert np.abs(got[i] - ref).max() <= RES_TOL


def test_pce_match_batch_matches_single_queries_and_oracle(ctx):
    rng = np.random.default_rng(77)
    n, C, H, W = 6, 3, 80, 112
    K = rng.normal(0, 0.01, size=(H, W))
    Iq = rng.uniform(40, 220, size=(n, C, H, W)).astype(np.float32)
    Wq = (K[None, None] * Iq * (np.arange(n) % 2)[:, None, None, None] +
          rng.normal(0, 0.7, size=(n, C, H, W))).astype(np.float32)  # odd queries carry K
    Kd = _dev(K.astype(np.float32))
    batch = ctx.pce_match_batch(Kd, _dev(Wq), _dev(Iq))
    for i in range(n):
        single = ctx.pce_match(Kd, _dev(Wq[i]), _dev(Iq[i]))
        r = O.pce_match(K, O.to_gray(Wq[i]), O.to_gray(Iq[i]))
        assert abs(batch[i][0] - r.pce) <= PCE_TOL * max(abs(r.pce), 1.0)
        assert abs(single[0] - batch[i][0]) <= 1e-6 * max(abs(batch[i][0]), 1.0)
        assert abs(batch[i][1] - r.ncc) <= 1e-4 * max(abs(r.ncc), 1e-3)
        assert (batch[i][0] > 60) == bool(i % 2)


def test_residual_of_an_unaligned_image_view(ctx):
    # a float image starting at an odd element offset (no 8-byte alignment)
    img = _frames(64, 96, 1, 1, seed=13)[0].transpose(2, 0, 1).astype(np.float32)
    buf = torch.zeros(img.size + 1, dtype=torch.float32, device="cuda")
    buf[1:] = _dev(img).reshape(-1)
    view = buf[1:].view(1, 64, 96)
    got = ctx.denoise_residual(view).cpu().numpy()
    assert np.abs(got - O.residual(img.astype(np.float64))).max() <= RES_TOL


@pytest.mark.parametrize("H,W,C,n", [(1080, 1920, 3, 4), (200, 328, 3, 3), (97, 250, 1, 2), (256, 256, 1, 1)])
def test_pce_from_images_matches_two_step_path_and_oracle(ctx, H, W, C, n):
    """prnu_pce_match_images (residuals never stored; grey synthesis of the
    combined noise for C = 3) against residual + pce_match_batch and, for the
    first query, the oracle."""
    cam = synth.Camera(H=H, W=W, C=C, camera_id=77)
    fr = synth.frames(cam, 16, device="cuda")
    num = torch.zeros((C, H, W), device="cuda")
    den = torch.zeros_like(num)
    ctx.fingerprint_accumulate(fr, 8, num, den)
    K = ctx.fingerprint_finalize(num, den, P.PRNU_TO_GRAY if C == 3 else 0)[0].clone()
    qf = torch.cat([synth.frames(cam, n - 1, stream=1, device="cuda"),
                    synth.frames(synth.foreign(cam), 1, stream=1, device="cuda")])
    q = ctx.sda_average(qf, 1)
    fused = ctx.pce_match_images(K, q)
    two = ctx.pce_match_batch(K, ctx.denoise_residual_batch(q), q)
    for (p1, c1, k1), (p2, c2, k2) in zip(fused, two):
        assert abs(p1 - p2) <= 1e-4 * max(abs(p2), 1.0)
        assert abs(c1 - c2) <= 1e-5 * max(abs(c2), 1e-3)
        assert k1 == k2 or abs(p2) < 60
    onum, oden = O.fingerprint_accumulate(fr.cpu().numpy(), 8)
    oK = O.fingerprint_finalize(onum, oden, O.TO_GRAY if C == 3 else 0)[0]
    qh = O.sda_average(qf[:1].cpu().numpy(), 1)[0]
    opce = O.pce_match(oK, O.to_gray(O.residual(qh)), O.to_gray(qh)).pce
    assert abs(fused[0][0] - opce) <= 1e-3 * abs(opce)


# 136 rows (factor 17): cuFFT correlation; 120 rows: the own-FFT passes
@pytest.mark.parametrize("H,W", [(136, 200), (120, 200)])
def test_pce_images_async_equals_sync_and_replays_in_a_graph(ctx, H, W):
    """prnu_pce_match_images_async leaves the same PCE / NCC / peak on the
    device as the synchronous call returns, and the whole step (accumulate,
    finalize, PCE) captured in a CUDA graph reproduces them on replay, also
    after its input frames are changed in place."""
    C, n = 3, 4
    cam = synth.Camera(H=H, W=W, C=C, camera_id=81)
    fr = synth.frames(cam, 12, device="cuda")
    qf = torch.cat([synth.frames(cam, n - 1, stream=1, device="cuda"),
                    synth.frames(synth.foreign(cam), 1, stream=1, device="cuda")])
    q = ctx.sda_average(qf, 1)
    num = torch.zeros((C, H, W), device="cuda")
    den = torch.zeros_like(num)
    flags = P.PRNU_TO_GRAY | P.PRNU_ZERO_MEAN | P.PRNU_WIENER_DFT
    out = (torch.full((n,), -1.0, dtype=torch.float64, device="cuda"),
           torch.full((n,), -1.0, dtype=torch.float64, device="cuda"),
           torch.full((n, 2), -1, dtype=torch.int32, device="cuda"))

    def step():
        num.zero_()
        den.zero_()
        ctx.fingerprint_accumulate(fr, 4, num, den)
        K = ctx.fingerprint_finalize(num, den, flags)
        ctx.pce_match_images_async(K[0], q, out=out)
        return K

    def sync_reference():
        num.zero_()
        den.zero_()
        ctx.fingerprint_accumulate(fr, 4, num, den)
        K = ctx.fingerprint_finalize(num, den, flags)
        return ctx.pce_match_images(K[0], q)

    def check(ref):
        pce, ncc, peak = out[0].cpu(), out[1].cpu(), out[2].cpu()
        for i, (p, c, k) in enumerate(ref):
            # same formula in double on the device and on the host
            assert abs(pce[i].item() - p) <= 1e-12 * max(abs(p), 1.0)
            assert abs(ncc[i].item() - c) <= 1e-12 * max(abs(c), 1e-6)
            assert tuple(peak[i].tolist()) == tuple(k)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    check(sync_reference())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        step()
    for v in out:
        v.fill_(-1)
    g.replay()
    torch.cuda.synchronize()
    check(sync_reference())
    fr.copy_(synth.frames(synth.foreign(cam), 12, device="cuda"))   # new frames, same buffer
    g.replay()
    torch.cuda.synchronize()
    ref = sync_reference()
    check(ref)
    assert abs(ref[0][0]) < 60 and abs(ref[-1][0]) > 60        # the foreign fingerprint now matches query n-1

    # the profiler's events inside a captured graph time each replay
    P.prnu_profile_reset(ctx.ctx)
    P.prnu_profile_enable(ctx.ctx, True)
    step()
    torch.cuda.synchronize()
    eager = {k: v for k, v in P.prnu_profile_read(ctx.ctx).items() if v[0] > 0}
    P.prnu_profile_reset(ctx.ctx)
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2, stream=s):
        step()
        step()
    P.prnu_profile_enable(ctx.ctx, False)
    g2.replay()
    torch.cuda.synchronize()
    captured = {k: v for k, v in P.prnu_profile_read(ctx.ctx).items() if v[0] > 0}
    del g2
    torch.cuda.synchronize()
    P.prnu_profile_reset(ctx.ctx)
    assert set(captured) == set(eager)
    for k, (nl, ms, nb) in captured.items():
        assert nl == 2 * eager[k][0] and nb == 2 * eager[k][2]
        assert ms > 0.0, k
    # with a selection only the named kernels are timed; all are counted
    P.prnu_profile_select(ctx.ctx, ["shrink", "sda_sum"])
    P.prnu_profile_enable(ctx.ctx, True)
    step()
    torch.cuda.synchronize()
    P.prnu_profile_enable(ctx.ctx, False)
    sel = {k: v for k, v in P.prnu_profile_read(ctx.ctx).items() if v[0] > 0}
    P.prnu_profile_reset(ctx.ctx)
    P.prnu_profile_select(ctx.ctx, None)
    assert set(sel) == set(eager)
    for k, (nl, ms, nb) in sel.items():
        assert nl == eager[k][0]
        assert (ms > 0.0) == (k in ("shrink", "sda_sum")), k
