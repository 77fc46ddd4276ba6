"""The fused group-sum + level-1 analysis kernel (prnu_params.sda_fusion):
the SDA frame of Sec. III-B and the first DWT level of the denoiser in one
pass over the frames.

Its arithmetic is the separate kernels' arithmetic in the same order on the
same exact integer sums, so the fingerprint sums must equal those of the
separate kernels bit for bit, and both match the FP64 oracle at the parity
tolerance.  Shapes cover whole and partial column blocks, the halo wrapping
to the row start, mirrored padding rows, several row strips, ragged last
groups, the longest group the packed 16-bit lanes allow (257 frames), one and
three channels and 16-bit subband storage; cases outside the kernel's
conditions (W not a multiple of 16, groups of 258 frames) take the separate
kernels and still match.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1909_04573_gb300 import prnu as P
from paper_1909_04573_gb300 import synth

pytestmark = pytest.mark.gpu

K_TOL = 1e-5


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_04573_gb300 import build
    build.build()
    c = P.Context(0)
    yield c
    c.close()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _accumulate(ctx, fr, d, fusion, dtype=P.PRNU_DTYPE_F32):
    C, H, W = fr.shape[3], fr.shape[1], fr.shape[2]
    num, den = torch.zeros((C, H, W), device="cuda"), torch.zeros((C, H, W), device="cuda")
    ctx.fingerprint_accumulate(fr, d, num, den, params=P.default_params(sda_fusion=fusion, dtype=dtype))
    torch.cuda.synchronize()
    return num.cpu().numpy(), den.cpu().numpy()


# (H, W, C, m, d, fusion): PRNU_SDA_FUSED = fused with the strips chosen per launch,
# n >= 1 = fused with n row strips, 0 = the default rule (fused for d >= 16)
CASES = [
    (64, 128, 3, 13, 5, P.PRNU_SDA_FUSED),     # whole column blocks, ragged last group (3 frames)
    (48, 1008, 3, 9, 4, P.PRNU_SDA_FUSED),     # partial last column block (504 output columns)
    (37, 48, 1, 12, 5, P.PRNU_SDA_FUSED),      # one channel, one partial block, mirrored rows (padded height 48)
    (100, 160, 3, 20, 10, 3),   # three row strips (re-summed 6-row halos)
    (30, 64, 3, 17, 17, 7),     # strips of 3 output rows: more strips than full iterations
    (32, 64, 3, 300, 257, 0),   # the longest group the 16-bit lanes hold, then a group of 43 (default rule)
    (1080, 1920, 3, 100, 50, 0),  # full HD, two SDA-50 groups (default rule)
]


@pytest.mark.parametrize("H,W,C,m,d,fusion", CASES)
def test_fused_equals_separate_bit_for_bit_and_matches_oracle(ctx, H, W, C, m, d, fusion):
    fr = synth.frames(synth.Camera(H=H, W=W, C=C, camera_id=H + W + m), m, drift_px=0.5)
    dev = fr.cuda()
    n_sep, d_sep = _accumulate(ctx, dev, d, P.PRNU_SDA_SEPARATE)
    n_fus, d_fus = _accumulate(ctx, dev, d, fusion)
    np.testing.assert_array_equal(n_fus, n_sep)
    np.testing.assert_array_equal(d_fus, d_sep)
    if H * W <= 200_000:
        onum, oden = O.fingerprint_accumulate(fr.numpy(), d)
        assert _rel(n_fus, onum) <= K_TOL and _rel(d_fus, oden) <= K_TOL
    else:  # full HD: the first group against the oracle
        onum, oden = O.fingerprint_accumulate(fr.numpy()[:d], d)
        n1, d1 = _accumulate(ctx, dev[:d].contiguous(), d, fusion)
        assert _rel(n1, onum) <= K_TOL and _rel(d1, oden) <= K_TOL


@pytest.mark.parametrize("dtype", [P.PRNU_DTYPE_F16, P.PRNU_DTYPE_BF16])
def test_fused_with_16bit_subbands(ctx, dtype):
    fr = synth.frames(synth.Camera(H=64, W=96, C=3, camera_id=31), 12).cuda()
    n_sep, d_sep = _accumulate(ctx, fr, 6, P.PRNU_SDA_SEPARATE, dtype)
    n_fus, d_fus = _accumulate(ctx, fr, 6, P.PRNU_SDA_FUSED, dtype)
    np.testing.assert_array_equal(n_fus, n_sep)
    np.testing.assert_array_equal(d_fus, d_sep)


@pytest.mark.parametrize("H,W,C,m,d", [(40, 52, 3, 9, 4), (32, 64, 3, 260, 258)])
def test_outside_the_fused_conditions(ctx, H, W, C, m, d):
    """W = 52 (rows not whole 16-byte chunks) and groups of 258 frames take
    the separate kernels even when fusion is asked for: same sums as forcing them."""
    fr = synth.frames(synth.Camera(H=H, W=W, C=C, camera_id=7), m).cuda()
    n0, d0 = _accumulate(ctx, fr, d, P.PRNU_SDA_FUSED)
    n1, d1 = _accumulate(ctx, fr, d, P.PRNU_SDA_SEPARATE)
    np.testing.assert_array_equal(n0, n1)
    np.testing.assert_array_equal(d0, d1)


def test_fused_in_a_cuda_graph(ctx):
    """The fused pass replays from a CUDA graph with the eager result."""
    H, W, C, m, d = 64, 128, 3, 20, 5
    fr = synth.frames(synth.Camera(H=H, W=W, C=C, camera_id=3), m).cuda()
    ref_n, ref_d = _accumulate(ctx, fr, d, P.PRNU_SDA_FUSED)
    prm = P.default_params(sda_fusion=P.PRNU_SDA_FUSED)
    f, mm, Hh, Ww, Cc, fs, rp = ctx._frames_geometry(fr)
    nb = P.prnu_workspace_size(ctx.ctx, H, W, C, prm, 4)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    num, den = torch.zeros((C, H, W), device="cuda"), torch.zeros((C, H, W), device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            num.zero_()
            den.zero_()
            P.prnu_fingerprint_accumulate(ctx.ctx, f.data_ptr(), m, H, W, C, fs, rp, d, prm, num.data_ptr(),
                                          den.data_ptr(), ws.data_ptr(), nb, side.cuda_stream)
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(2):
        num.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(num.cpu().numpy(), ref_n)
        np.testing.assert_array_equal(den.cpu().numpy(), ref_d)


def test_invalid_fusion_setting(ctx):
    fr = synth.frames(synth.Camera(H=32, W=64, C=3, camera_id=1), 4).cuda()
    num, den = torch.zeros((3, 32, 64), device="cuda"), torch.zeros((3, 32, 64), device="cuda")
    for bad in (-3, 257):
        with pytest.raises(P.PrnuError) as e:
            ctx.fingerprint_accumulate(fr, 2, num, den, params=P.default_params(sda_fusion=bad))
        assert e.value.status == P.PRNU_EINVAL


def test_fused_in_multi_camera_passes(ctx):
    """prnu_fingerprint_accumulate_multi: groups of several cameras in one
    pass (per-group frame descriptors, ragged counts), the geometries the
    fused kernel serves and one it does not (W = 52): the same sums as the
    separate kernels, bit for bit, and the oracle's."""
    specs = [(64, 96, 3, 13, 4), (64, 96, 3, 9, 9), (48, 128, 1, 11, 3), (40, 52, 3, 7, 2), (64, 96, 3, 20, 7)]
    frames = [synth.frames(synth.Camera(H=H, W=W, C=C, camera_id=900 + i), m, drift_px=0.3)
              for i, (H, W, C, m, d) in enumerate(specs)]
    res = {}
    for fusion in (P.PRNU_SDA_FUSED, P.PRNU_SDA_SEPARATE):  # multi-camera passes fuse only when asked
        items = []
        for fr, (H, W, C, m, d) in zip(frames, specs):
            items.append((fr.cuda(), d, torch.zeros((C, H, W), device="cuda"), torch.zeros((C, H, W), device="cuda")))
        ctx.fingerprint_accumulate_multi(items, params=P.default_params(sda_fusion=fusion), groups_per_pass=5)
        torch.cuda.synchronize()
        res[fusion] = [(n.cpu().numpy(), dd.cpu().numpy()) for _, _, n, dd in items]
    for (nf, df), (ns, ds) in zip(res[P.PRNU_SDA_FUSED], res[P.PRNU_SDA_SEPARATE]):
        np.testing.assert_array_equal(nf, ns)
        np.testing.assert_array_equal(df, ds)
    for fr, (H, W, C, m, d), (nf, df) in zip(frames, specs, res[P.PRNU_SDA_FUSED]):
        onum, oden = O.fingerprint_accumulate(fr.numpy(), d)
        assert _rel(nf, onum) <= K_TOL and _rel(df, oden) <= K_TOL
