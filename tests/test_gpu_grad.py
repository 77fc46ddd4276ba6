"""Adjoint kernels of the differentiable chain against the FP64 oracle adjoint
(oracle/grad.py) and against central differences of the CUDA forward (GPU).

Tolerances: the CUDA chain runs in float32; per-step adjoints agree with the
FP64 adjoint to a relative L2 error of 1e-4 (residual, PCE: a few hundred
float32 operations per value, errors ~1e-6 each), weight and sigma0
gradients of the whole chain to 1e-3 (they are sums of 10^5..10^6 such
terms).  Central differences of the float32 forward with h = 1e-3 carry a
truncation error (kinks of the min-window choice, curvature) bounded here by
2e-2 of the derivative, plus the forward's rounding, about 1e-6 |J| / h."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import grad as OG
from paper_1909_04573_gb300 import grad as G
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


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _np(t):
    return t.detach().double().cpu().numpy()


def _sig(v=3.0):
    return torch.tensor(v, dtype=torch.float64, requires_grad=True)


@pytest.mark.parametrize("m,H,W,C,d", [(37, 48, 80, 3, 8), (16, 64, 64, 1, 16), (5, 16, 4100, 1, 2)])
def test_sda_weighted_and_backward_match_oracle(ctx, m, H, W, C, d):
    fr = synth.frames(synth.Camera(H=H, W=W, C=C, camera_id=60), m, device="cuda")
    rng = np.random.default_rng(0)
    w = torch.tensor(rng.uniform(0.02, 0.2, m), dtype=torch.float32, device="cuda", requires_grad=True)
    S = G.sda_weighted(fr, w, d, ctx)
    frn = fr.cpu().numpy()
    assert _rel(_np(S), OG.sda_weighted(frn, _np(w), d)) <= 1e-6
    gS = torch.tensor(rng.standard_normal(S.shape), dtype=torch.float32, device="cuda")
    S.backward(gS)
    assert _rel(_np(w.grad), OG.sda_weighted_vjp(frn, d, _np(gS))) <= 1e-5


def test_equal_weights_give_the_sda_mean(ctx):
    fr = synth.frames(synth.Camera(H=40, W=48, C=3, camera_id=61), 20, device="cuda")
    w = torch.full((20,), 1.0 / 8, device="cuda")
    w[16:] = 1.0 / 4
    S = G.sda_weighted(fr, w, 8, ctx)
    assert _rel(_np(S), O.sda_average(fr.cpu().numpy(), 8)) <= 1e-6


def test_residual_ckpt_forward_is_the_residual(ctx):
    img = ctx.sda_average(synth.frames(synth.Camera(H=64, W=96, C=3, camera_id=62), 6, device="cuda"), 3)
    W = G.residual(img, _sig(), ctx)
    torch.cuda.synchronize()
    assert torch.equal(W, ctx.denoise_residual_batch(img))


@pytest.mark.parametrize("n,C,H,W,levels,s0", [(2, 1, 64, 96, 4, 3.0), (1, 3, 128, 64, 4, 3.0), (3, 1, 32, 48, 3, 2.0),
                                              (1, 1, 256, 256, 4, 3.0)])
def test_residual_backward_matches_oracle(ctx, n, C, H, W, levels, s0):
    img = ctx.sda_average(synth.frames(synth.Camera(H=H, W=W, C=C, camera_id=63), 2 * n, device="cuda"), 2)
    img.requires_grad_(True)
    sig = _sig(s0)
    Wr = G.residual(img, sig, ctx, levels)
    rng = np.random.default_rng(1)
    gW = torch.tensor(rng.standard_normal(Wr.shape), dtype=torch.float32, device="cuda")
    Wr.backward(gW)
    prm = O.Params(levels=levels)
    for i in range(n):
        ow, cache = OG.residual_forward(_np(img[i]), s0, prm)
        assert float(np.abs(_np(Wr[i]) - ow).max()) <= 1e-3
        og, _ = OG.residual_vjp(cache, _np(gW[i]))
        assert _rel(_np(img.grad[i]), og) <= 1e-4
    og_s = sum(OG.residual_vjp(OG.residual_forward(_np(img[i]), s0, prm)[1], _np(gW[i]))[1] for i in range(n))
    assert abs(float(sig.grad) - og_s) <= 1e-4 * abs(og_s)


@pytest.mark.parametrize("gray,C", [(True, 3), (False, 3), (True, 1)])
def test_mle_images_and_backward_match_oracle(ctx, gray, C):
    rng = np.random.default_rng(2)
    n, H, W = 4, 24, 40
    S = torch.tensor(rng.uniform(20, 230, (n, C, H, W)), dtype=torch.float32, device="cuda", requires_grad=True)
    Wr = torch.tensor(rng.standard_normal((n, C, H, W)), dtype=torch.float32, device="cuda", requires_grad=True)
    K = G.mle(Wr, S, ctx, gray=gray)
    oK, cache = OG.mle_forward(_np(Wr), _np(S), gray)
    assert _rel(_np(K), oK) <= 1e-6
    gK = torch.tensor(rng.standard_normal(K.shape), dtype=torch.float32, device="cuda")
    K.backward(gK)
    ogW, ogS = OG.mle_vjp(cache, _np(gK))
    assert _rel(_np(Wr.grad), ogW) <= 1e-6 and _rel(_np(S.grad), ogS) <= 1e-6


@pytest.mark.parametrize("C,per_query", [(1, False), (3, False), (3, True)])
def test_pce_backward_matches_oracle(ctx, C, per_query):
    rng = np.random.default_rng(3)
    n, H, W = 3, 96, 128
    Kn = rng.standard_normal((n, H, W) if per_query else (H, W)) * 0.01
    Iq = rng.uniform(40, 220, (n, C, H, W))
    Kb = Kn if per_query else np.broadcast_to(Kn, (n, H, W))
    Wq = 0.5 * Kb[:, None] * Iq + rng.standard_normal((n, C, H, W))
    K = torch.tensor(Kn, dtype=torch.float32, device="cuda", requires_grad=True)
    Wt = torch.tensor(Wq, dtype=torch.float32, device="cuda", requires_grad=True)
    It = torch.tensor(Iq, dtype=torch.float32, device="cuda")
    p = G.pce(K, Wt, It, ctx, nbhd=11)
    g = torch.tensor(rng.uniform(0.5, 1.5, n), dtype=torch.float64, device="cuda")
    p.backward(g)
    gK = np.zeros_like(Kn)
    for q in range(n):
        val, cache = OG.pce_forward(Kb[q], Wq[q], Iq[q], 11)
        assert abs(p[q].item() - val) <= 1e-3 * abs(val)
        gk, gw = OG.pce_vjp(cache, float(g[q]))
        assert _rel(_np(Wt.grad[q]), gw) <= 1e-4
        if per_query:
            assert _rel(_np(K.grad[q]), gk) <= 1e-4
        else:
            gK += gk
    if not per_query:
        assert _rel(_np(K.grad), gK) <= 1e-4


def _diff_case(m, H, W, d, nq, cid):
    cam = synth.Camera(H=H, W=W, C=1, camera_id=cid)
    fr = synth.frames(cam, m, device="cuda")
    q = synth.frames(cam, nq, stream=1, device="cuda")
    return fr, q


def test_chain_gradient_matches_oracle_and_central_differences(ctx):
    m, H, W, d, nq = 32, 128, 128, 8, 2
    fr, qf = _diff_case(m, H, W, d, nq, 64)
    qimg = ctx.sda_average(qf, 1)
    w = torch.full((m,), 1.0 / d, device="cuda", requires_grad=True)
    sig = _sig()
    J = G.mean_pce(fr, w, d, sig, qimg, ctx)
    J.backward()
    oJ, ogw, ogs = OG.objective_and_grad(fr.cpu().numpy(), d, np.full(m, 1.0 / d), 3.0, _np(qimg))
    assert abs(J.item() - oJ) <= 1e-3 * abs(oJ)
    assert _rel(_np(w.grad), ogw) <= 1e-3
    assert abs(float(sig.grad) - ogs) <= 1e-3 * abs(ogs)
    # central differences of the CUDA forward, h = 1e-3, along sigma0 and along
    # the normalised weight gradient (the direction of largest signal); the
    # float32 forward's rounding adds up to ~1e-6 |J| / h to a difference quotient
    h = 1e-3
    noise = 4e-6 * abs(J.item()) / h
    with torch.no_grad():
        f = lambda ww, s: G.mean_pce(fr, ww, d, torch.tensor(s, dtype=torch.float64), qimg, ctx).item()
        fd_s = (f(w, 3.0 + h) - f(w, 3.0 - h)) / (2 * h)
        u = w.grad / w.grad.norm()
        fd_u = (f(w + h * u, 3.0) - f(w - h * u, 3.0)) / (2 * h)
    assert abs(fd_s - float(sig.grad)) <= 2e-2 * abs(float(sig.grad)) + noise
    gn = float(w.grad.norm())
    assert abs(fd_u - gn) <= 2e-2 * gn + noise


def test_full_size_differentiation_workload_matches_oracle(ctx):
    """256 grey 512x512 frames, SDA groups of 16 with weights 1/16, 2 queries."""
    m, H, W, d, nq = 256, 512, 512, 16, 2
    fr, qf = _diff_case(m, H, W, d, nq, 65)
    qimg = ctx.sda_average(qf, 1)
    w = torch.full((m,), 1.0 / d, device="cuda", requires_grad=True)
    sig = _sig()
    J = G.mean_pce(fr, w, d, sig, qimg, ctx)
    J.backward()
    oJ, ogw, ogs = OG.objective_and_grad(fr.cpu().numpy(), d, np.full(m, 1.0 / d), 3.0, _np(qimg))
    assert oJ > 60
    assert abs(J.item() - oJ) <= 1e-3 * abs(oJ)
    assert _rel(_np(w.grad), ogw) <= 1e-3
    assert abs(float(sig.grad) - ogs) <= 1e-3 * abs(ogs)


def test_gradient_entry_points_reject_unsupported_inputs(ctx):
    with pytest.raises(P.PrnuError) as e:
        P.prnu_workspace_size_grad(ctx.ctx, 1080, 1920, 3, P.default_params(), 1)
    assert e.value.status == P.PRNU_EUNSUPPORTED
    with pytest.raises(P.PrnuError) as e:
        P.prnu_workspace_size_grad(ctx.ctx, 64, 64, 1, P.default_params(dtype=P.PRNU_DTYPE_F16), 1)
    assert e.value.status == P.PRNU_EUNSUPPORTED
