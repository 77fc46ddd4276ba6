"""The level-1 MLE step in its two tilings (tuner kind 3): the 58 x 32 wide
tile, whose 32 coefficient columns keep every lane of the column synthesis
busy, and the 32 x 32 tile.  Both take the same operations in the same order
(column synthesis, row synthesis, then W I and I I image by image, Sec.
III-A), so num/den must be identical bit for bit, with plain and compensated
sums, ragged crops (tiles past the right and bottom edges, the periodic wrap
of the first and last tiles) and multi-camera passes; the wide tile matches
the FP64 oracle.  Geometries outside the wide tile's conditions (odd W,
16-bit subbands) take the 32 x 32 tile under every choice."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1909_04573_gb300 import prnu as P
from paper_1909_04573_gb300 import synth

pytestmark = pytest.mark.gpu

WIDE, TILE = 1, 2


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_04573_gb300 import build
    build.build()
    c = P.Context(0)
    yield c
    c.close()


def _accumulate(ctx, fr, d, prm, choice, comp=False):
    m, H, W, C = fr.shape
    ctx.autotune_level(H, W, 3, 1, choice, prm)
    shape = (2, C, H, W) if comp else (C, H, W)
    num, den = torch.zeros(shape, device="cuda"), torch.zeros(shape, device="cuda")
    ctx.fingerprint_accumulate(fr, d, num, den, params=prm)
    torch.cuda.synchronize()
    ctx.autotune_level(H, W, 3, 1, -1, prm)
    return num, den


@pytest.mark.parametrize("H,W,C,m,d,dtype,comp", [
    (1080, 1920, 3, 60, 20, P.PRNU_DTYPE_F32, False),   # the video geometry, three groups
    (1080, 1920, 1, 30, 10, P.PRNU_DTYPE_F32, True),    # compensated sums
    (201, 334, 3, 13, 4, P.PRNU_DTYPE_F32, False),      # partial last tiles in both directions, ragged group
    (48, 116, 3, 7, 3, P.PRNU_DTYPE_F32, True),         # exactly two tiles wide
    (40, 52, 3, 5, 2, P.PRNU_DTYPE_F32, False),         # one tile wider than the image
    (201, 333, 3, 9, 4, P.PRNU_DTYPE_F32, False),       # odd W: the 32 x 32 tile under both choices
    (97, 250, 1, 9, 9, P.PRNU_DTYPE_F16, False),        # 16-bit subbands: likewise
])
def test_wide_and_square_tiles_give_identical_sums(ctx, H, W, C, m, d, dtype, comp):
    prm = P.default_params(dtype=dtype, compensated=comp)
    fr = synth.frames(synth.Camera(H=H, W=W, C=C, camera_id=H + W + m), m, drift_px=0.4, device="cuda")
    nw, dw = _accumulate(ctx, fr, d, prm, WIDE, comp)
    nt, dt = _accumulate(ctx, fr, d, prm, TILE, comp)
    assert torch.equal(nw, nt) and torch.equal(dw, dt)
    hi = dw[0] if comp else dw  # the low parts of compensated sums take either sign
    assert bool(torch.isfinite(nw).all()) and bool((hi >= 0).all()) and float(hi.sum()) > 0


def test_wide_tile_matches_the_oracle(ctx):
    H, W, C, m, d = 64, 136, 3, 11, 4
    fr = synth.frames(synth.Camera(H=H, W=W, C=C, camera_id=77), m, drift_px=0.3)
    n, dd = _accumulate(ctx, fr.cuda(), d, P.default_params(), WIDE)
    onum, oden = O.fingerprint_accumulate(fr.numpy(), d)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    assert rel(n.cpu().numpy(), onum) <= 1e-5 and rel(dd.cpu().numpy(), oden) <= 1e-5


def test_wide_tile_in_multi_camera_passes(ctx):
    """Groups of three cameras in one pass: the wide tile flushes its register
    sums when the camera changes, as the square tile does."""
    specs = [(120, 232, 3, 9, 4), (120, 232, 3, 7, 7), (120, 232, 3, 12, 5)]
    frames = [synth.frames(synth.Camera(H=H, W=W, C=C, camera_id=500 + i), mm, device="cuda")
              for i, (H, W, C, mm, d) in enumerate(specs)]
    prm = P.default_params()
    res = {}
    for choice in (WIDE, TILE):
        ctx.autotune_level(120, 232, 3, 1, choice, prm)
        items = [(fr, d, torch.zeros((C, H, W), device="cuda"), torch.zeros((C, H, W), device="cuda"))
                 for fr, (H, W, C, mm, d) in zip(frames, specs)]
        ctx.fingerprint_accumulate_multi(items, params=prm, groups_per_pass=6)
        torch.cuda.synchronize()
        res[choice] = [(n.clone(), dd.clone()) for _, _, n, dd in items]
    ctx.autotune_level(120, 232, 3, 1, -1, prm)
    for (nw, dw), (nt, dt) in zip(res[WIDE], res[TILE]):
        assert torch.equal(nw, nt) and torch.equal(dw, dt)


def test_mle_step_choice_bounds(ctx):
    prm = P.default_params()
    assert ctx.autotune_level(64, 64, 3, 1, -2, prm) == 0
    for bad_level in (0, 2):
        with pytest.raises(P.PrnuError):
            ctx.autotune_level(64, 64, 3, bad_level, 1, prm)
    with pytest.raises(P.PrnuError):
        ctx.autotune_level(64, 64, 3, 1, 3, prm)
