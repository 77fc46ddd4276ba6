"""The autotuner's launch choices: every level-1 analysis shape, every
analysis form of levels 2.. and every synthesis form give bit-identical
results, the two shrink forms agree to float32 rounding, and the tuner's
choices are cached and used (GPU)."""
import pytest
import torch

from paper_1909_04573_gb300 import prnu as P
from paper_1909_04573_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_04573_gb300 import build
    build.build()
    c = P.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("H,W,C,dtype", [(200, 328, 3, P.PRNU_DTYPE_F32), (1080, 1920, 3, P.PRNU_DTYPE_F32),
                                         (97, 250, 1, P.PRNU_DTYPE_F16), (256, 256, 1, P.PRNU_DTYPE_BF16)])
def test_every_shape_gives_identical_residuals(ctx, H, W, C, dtype):
    prm = P.default_params(dtype=dtype)
    img = ctx.sda_average(synth.frames(synth.Camera(H=H, W=W, C=C, camera_id=41), 3, device="cuda"), 3)[0]
    ctx.autotune_set(H, W, -1, prm)
    ref = ctx.denoise_residual(img, params=prm).clone()
    for s in range(len(P.STREAM_SHAPES)):
        ctx.autotune_set(H, W, s, prm)
        out = ctx.denoise_residual(img, params=prm)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), f"shape {P.STREAM_SHAPES[s]}"
    ctx.autotune_set(H, W, -1, prm)


def test_tuner_picks_a_shape_and_keeps_results(ctx):
    H, W, C = 1080, 1920, 3
    fr = synth.frames(synth.Camera(H=H, W=W, C=C, camera_id=42), 20, device="cuda")
    num0, den0 = torch.zeros((C, H, W), device="cuda"), torch.zeros((C, H, W), device="cuda")
    ctx.autotune_set(H, W, -1)
    ctx.fingerprint_accumulate(fr, 5, num0, den0)
    shape, ms = ctx.autotune(H, W, C, images=4)
    assert shape in P.STREAM_SHAPES and 0 < ms < 100
    num1, den1 = torch.zeros_like(num0), torch.zeros_like(den0)
    ctx.fingerprint_accumulate(fr, 5, num1, den1)
    torch.cuda.synchronize()
    # the level-1 shapes and the analysis / synthesis choices are bit-identical;
    # a shrink choice sums the windows in another order (float32 rounding)
    assert torch.equal(den0, den1)
    assert float((num1 - num0).norm() / num0.norm()) <= 1e-6
    ctx.autotune_set(H, W, -1)


def test_invalid_shape_is_rejected(ctx):
    with pytest.raises(P.PrnuError) as e:
        ctx.autotune_set(64, 64, len(P.STREAM_SHAPES))
    assert e.value.status == P.PRNU_EINVAL
    with pytest.raises(P.PrnuError):
        ctx.autotune(64, 64, 2)                                   # C must be 1 or 3


@pytest.mark.parametrize("H,W,C,dtype", [(200, 328, 3, P.PRNU_DTYPE_F32), (1080, 1920, 1, P.PRNU_DTYPE_F32),
                                         (97, 250, 1, P.PRNU_DTYPE_F16)])
def test_per_level_choices(ctx, H, W, C, dtype):
    """Every per-level launch choice the tuner may pin: the analysis and the
    synthesis forms give bit-identical residuals; the two shrink forms sum the
    windows in different orders and agree to float32 rounding."""
    prm = P.default_params(dtype=dtype)
    img = ctx.sda_average(synth.frames(synth.Camera(H=H, W=W, C=C, camera_id=43), 3, device="cuda"), 3)[0]
    ctx.autotune_set(H, W, -1, prm)
    ref = ctx.denoise_residual(img, params=prm).clone()
    for kind, levels, nch, exact in ((0, range(2, 5), 3, True), (2, range(2, 5), 3, True), (1, range(1, 5), 2, False)):
        for level in levels:
            for c in range(nch):
                assert ctx.autotune_level(H, W, kind, level, c, prm) == c
                out = ctx.denoise_residual(img, params=prm)
                torch.cuda.synchronize()
                if exact:
                    assert torch.equal(out, ref), (kind, level, c)
                else:
                    assert float((out - ref).abs().max()) <= 1e-4 * max(1.0, float(ref.abs().max())), (kind, level, c)
            ctx.autotune_level(H, W, kind, level, -1, prm)
    ctx.autotune_set(H, W, -1, prm)


def test_tuner_sets_every_level(ctx):
    H, W, C = 272, 480, 3
    prm = P.default_params()
    img = ctx.sda_average(synth.frames(synth.Camera(H=H, W=W, C=C, camera_id=44), 2, device="cuda"), 2)[0]
    ctx.autotune_set(H, W, -1, prm)
    ref = ctx.denoise_residual(img, params=prm).clone()
    ctx.autotune(H, W, C, prm, images=2)
    got = {(k, l): ctx.autotune_level(H, W, k, l) for k, ls in ((0, range(2, 5)), (1, range(1, 5)), (2, range(2, 5)))
           for l in ls}
    assert all(0 <= v < (2 if k == 1 else 3) for (k, _), v in got.items())
    out = ctx.denoise_residual(img, params=prm)
    torch.cuda.synchronize()
    assert float((out - ref).abs().max()) <= 1e-4 * max(1.0, float(ref.abs().max()))
    with pytest.raises(P.PrnuError):
        ctx.autotune_level(H, W, 0, 1, 0)       # no analysis choice at level 1
    with pytest.raises(P.PrnuError):
        ctx.autotune_level(H, W, 1, 5, 0)       # past the last level
    ctx.autotune_set(H, W, -1, prm)
