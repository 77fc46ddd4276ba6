"""Sanitizer substitutes (GPU): the debug build's device-side index checks and
guard-band canaries around every output buffer.

The debug build (libprnu_debug.so, the same sources compiled with PRNU_DEBUG)
checks the global-memory indices of its kernels and records the first failure
per source file instead of trapping.  Each entry-point family runs here on
small ragged shapes through that build: its results must match the FP64
oracle at the parity tolerances and prnu_debug_status must report no failed
check.  Every output buffer sits between two guard bands filled with a
sentinel bit pattern, checked untouched after the call, in the debug and in
the release build.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1909_04573_gb300 import prnu as P
from paper_1909_04573_gb300 import synth

pytestmark = pytest.mark.gpu

GUARD = 4096                # floats on each side of an output
SENTINEL = 0x7FC0DEAD       # a quiet-NaN bit pattern no kernel writes


@pytest.fixture(scope="module", params=["debug", "release"])
def lib_ctx(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_04573_gb300 import build
    build.build()
    if request.param == "debug":
        P.set_library(build.build(debug=True))
    ctx = P.Context(0)
    yield request.param, ctx
    ctx.close()
    P.set_library(None)


class Guarded:
    """A float32 (or float64 / int32) tensor of `shape` inside a buffer with
    GUARD elements of sentinel on each side."""

    def __init__(self, shape, dtype=torch.float32, fill=None):
        n = int(np.prod(shape))
        self.buf = torch.empty(n + 2 * GUARD, dtype=dtype, device="cuda")
        self.buf.view(torch.int32 if dtype.itemsize == 4 else torch.int64).fill_(SENTINEL)
        self.t = self.buf[GUARD:GUARD + n].view(shape)
        if fill is not None:
            self.t.fill_(fill)

    def intact(self):
        iv = self.buf.view(torch.int32 if self.buf.dtype.itemsize == 4 else torch.int64)
        return bool((iv[:GUARD] == SENTINEL).all()) and bool((iv[-GUARD:] == SENTINEL).all())


def _check(lib, ctx):
    torch.cuda.synchronize()
    st, where = P.prnu_debug_status(ctx.ctx)
    if lib == "debug":
        assert st == P.PRNU_OK, where
    else:
        assert st == P.PRNU_EUNSUPPORTED


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_sda_average(lib_ctx):
    lib, ctx = lib_ctx
    fr = np.random.default_rng(7).integers(0, 256, size=(11, 37, 50, 3), dtype=np.uint8)
    f, m, H, W, C, fs, rp = ctx._frames_geometry(torch.as_tensor(fr).cuda())
    out = Guarded((3, C, H, W))
    P.prnu_sda_average(ctx.ctx, f.data_ptr(), m, H, W, C, fs, rp, 4, out.t.data_ptr(), ctx._stream())
    _check(lib, ctx)
    np.testing.assert_array_equal(out.t.cpu().numpy(), O.sda_average(fr, 4).astype(np.float32))
    assert out.intact()


@pytest.mark.parametrize("H,W,C", [(37, 50, 3), (64, 64, 1), (100, 300, 1)])
def test_residual(lib_ctx, H, W, C):
    lib, ctx = lib_ctx
    img = synth.frames(synth.Camera(H=H, W=W, C=C, camera_id=H), 1)[0].permute(2, 0, 1).float().contiguous()
    out = Guarded((C, H, W))
    ctx.denoise_residual(img.cuda(), out=out.t)
    _check(lib, ctx)
    assert float(np.abs(out.t.cpu().numpy() - O.residual(img.numpy().astype(np.float64))).max()) <= 1e-3
    assert out.intact()


@pytest.mark.parametrize("pipeline,H,W", [(0, 40, 52), (2, 40, 52), (0, 48, 64)])  # 48 x 64: fused group sums
def test_accumulate_and_finalize(lib_ctx, pipeline, H, W):
    lib, ctx = lib_ctx
    C, m, d = 3, 17, 5
    fr = synth.frames(synth.Camera(H=H, W=W, C=C, camera_id=5), m, drift_px=1.0)
    num, den = Guarded((C, H, W), fill=0.0), Guarded((C, H, W), fill=0.0)
    prm = P.default_params(pipeline_passes=pipeline, sda_fusion=P.PRNU_SDA_FUSED if W == 64 else 0)
    ctx.fingerprint_accumulate(fr.cuda(), d, num.t, den.t, params=prm, images_per_pass=2)
    _check(lib, ctx)
    onum, oden = O.fingerprint_accumulate(fr.numpy(), d)
    assert _rel(num.t.cpu().numpy(), onum) <= 1e-5 and _rel(den.t.cpu().numpy(), oden) <= 1e-5
    assert num.intact() and den.intact()
    flags = P.PRNU_TO_GRAY | P.PRNU_ZERO_MEAN | P.PRNU_WIENER_DFT
    K = Guarded((1, H, W))
    n = P.prnu_workspace_size(ctx.ctx, H, W, C, prm, 1)
    ws = ctx.workspace(n)
    P.prnu_fingerprint_finalize(ctx.ctx, num.t.data_ptr(), den.t.data_ptr(), H, W, C, flags, prm, K.t.data_ptr(),
                                ws.data_ptr(), ws.numel(), ctx._stream())
    _check(lib, ctx)
    oK = O.fingerprint_finalize(onum, oden, O.TO_GRAY | O.ZERO_MEAN | O.WIENER_DFT)
    assert _rel(K.t.cpu().numpy(), oK) <= 1e-5
    assert K.intact()


def test_multi_camera_and_persistent(lib_ctx):
    lib, ctx = lib_ctx
    specs = [(64, 96, 3, 13, 4), (80, 112, 1, 25, 3), (37, 50, 3, 9, 2)]
    for persistent in (False, True):
        items, guards = [], []
        for i, (H, W, C, m, d) in enumerate(specs):
            fr = synth.frames(synth.Camera(H=H, W=W, C=C, camera_id=500 + i), m, device="cuda")
            num, den = Guarded((C, H, W), fill=0.0), Guarded((C, H, W), fill=0.0)
            guards += [num, den]
            items.append((fr, d, num.t, den.t))
        if persistent:
            ctx.fingerprint_accumulate_persistent(items)
        else:  # the fused group-sum kernel where a geometry allows it
            ctx.fingerprint_accumulate_multi(items, params=P.default_params(sda_fusion=P.PRNU_SDA_FUSED))
        _check(lib, ctx)
        for fr, d, n, dd in items:
            onum, oden = O.fingerprint_accumulate(fr.cpu().numpy(), d)
            assert _rel(n.cpu().numpy(), onum) <= 1e-5 and _rel(dd.cpu().numpy(), oden) <= 1e-5
        assert all(g.intact() for g in guards)


@pytest.mark.parametrize("H,W", [(96, 80), (74, 94)])  # own FFT; a geometry on cuFFT
def test_pce_paths(lib_ctx, H, W):
    lib, ctx = lib_ctx
    cam = synth.Camera(H=H, W=W, C=3, camera_id=600 + H)
    fr = synth.frames(cam, 24, device="cuda")
    num, den = torch.zeros((3, H, W), device="cuda"), torch.zeros((3, H, W), device="cuda")
    ctx.fingerprint_accumulate(fr, 8, num, den)
    K = ctx.fingerprint_finalize(num, den, P.PRNU_TO_GRAY)[0].contiguous()
    q = ctx.sda_average(synth.frames(cam, 2, stream=1, device="cuda"), 1)
    wq = Guarded(tuple(q.shape))
    ctx.denoise_residual_batch(q, out=wq.t)
    two = ctx.pce_match_batch(K, wq.t, q)
    outs = (Guarded((2,), torch.float64), Guarded((2,), torch.float64), Guarded((2, 2), torch.int32))
    ctx.pce_match_images_async(K, q, out=tuple(g.t for g in outs))
    _check(lib, ctx)
    for i in range(2):
        r = O.pce_match(K.cpu().numpy().astype(np.float64), O.to_gray(wq.t[i].cpu().numpy().astype(np.float64)),
                        O.to_gray(q[i].cpu().numpy().astype(np.float64)))
        assert abs(two[i][0] - r.pce) <= 1e-3 * abs(r.pce)
        assert abs(outs[0].t[i].item() - r.pce) <= 1e-3 * abs(r.pce)
    assert wq.intact() and all(g.intact() for g in outs)
