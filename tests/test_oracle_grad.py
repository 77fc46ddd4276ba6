"""Pins of the FP64 oracle adjoint (oracle/grad.py), no GPU.

Every vector-Jacobian product is checked against FP64 central differences of
the oracle's forward (itself pinned by the other oracle tests), plus closed
forms: the shrink with every window mean below sigma0^2 is the identity; the
residual is then a linear orthogonal projection, so its adjoint is itself; and
PCE is invariant to scaling K, to scaling W_q and to adding a constant to W_q,
so its gradient is orthogonal to K, to W_q and to the constant field."""
import numpy as np
import pytest

import oracle as O
from oracle import grad as G


def _fd(f, x, v, h):
    return (f(x + h * v) - f(x - h * v)) / (2 * h)


def _scene(rng, shape, sigma=2.0):
    H, W = shape[-2:]
    white = rng.standard_normal(shape)
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.fftfreq(W)[None, :]
    gain = np.exp(-2 * np.pi ** 2 * sigma ** 2 * (fx * fx + fy * fy))
    return np.real(np.fft.ifft2(np.fft.fft2(white) * gain)) * 60 + 128


def test_shrink_vjp_matches_central_differences():
    rng = np.random.default_rng(0)
    c = rng.standard_normal((16, 20)) * 4.0
    gn = rng.standard_normal(c.shape)
    v = rng.standard_normal(c.shape)
    _, cache = G.shrink_forward(c, 3.0)
    gc, gs = G.shrink_vjp(cache, gn)
    f = lambda x: float(np.sum(gn * G.shrink_forward(x, 3.0)[0]))
    assert abs(_fd(f, c, v, 1e-6) - float(np.sum(gc * v))) <= 1e-7 * max(1.0, abs(float(np.sum(gc * v))))
    fs = lambda s: float(np.sum(gn * G.shrink_forward(c, s)[0]))
    assert abs((fs(3.0 + 1e-6) - fs(3.0 - 1e-6)) / 2e-6 - gs) <= 1e-6 * max(1.0, abs(gs))


def test_shrink_below_noise_floor_is_identity():
    rng = np.random.default_rng(1)
    c = rng.uniform(-1.0, 1.0, (12, 12))          # every window mean of c^2 < 1 < sigma0^2
    n, cache = G.shrink_forward(c, 3.0)
    np.testing.assert_allclose(n, c, rtol=1e-15)             # c s2 / s2, one rounding
    gn = rng.standard_normal(c.shape)
    gc, gs = G.shrink_vjp(cache, gn)
    np.testing.assert_allclose(gc, gn, rtol=1e-15)
    assert gs == 0.0


@pytest.mark.parametrize("shape,levels", [((1, 32, 32), 3), ((1, 40, 56), 3), ((3, 32, 48), 4)])
def test_residual_vjp_matches_central_differences(shape, levels):
    rng = np.random.default_rng(2)
    prm = O.Params(levels=levels)
    img = _scene(rng, shape)
    gW = rng.standard_normal(shape)
    v = rng.standard_normal(shape)
    _, cache = G.residual_forward(img, 3.0, prm)
    gimg, gs = G.residual_vjp(cache, gW)
    f = lambda x: float(np.sum(gW * G.residual_forward(x, 3.0, prm)[0]))
    want = float(np.sum(gimg * v))
    assert abs(_fd(f, img, v, 1e-5) - want) <= 1e-6 * max(1.0, abs(want))
    fs = lambda s: float(np.sum(gW * G.residual_forward(img, s, prm)[0]))
    assert abs((fs(3.0 + 1e-6) - fs(3.0 - 1e-6)) / 2e-6 - gs) <= 1e-5 * max(1.0, abs(gs))


def test_residual_forward_equals_pipeline_noise_form():
    rng = np.random.default_rng(3)
    img = _scene(rng, (3, 40, 56))
    np.testing.assert_allclose(G.residual_forward(img, 3.0)[0], O.residual_noise_form(img), atol=1e-10)


def test_linear_residual_is_self_adjoint():
    """sigma0 so large that every coefficient is kept as noise: W = x - P_L x
    with P_L the orthogonal projection on the coarse space, so R^T = R."""
    rng = np.random.default_rng(4)
    x = rng.standard_normal((1, 32, 32))
    gW = rng.standard_normal((1, 32, 32))
    _, cache = G.residual_forward(x, 1e4)
    gimg, gs = G.residual_vjp(cache, gW)
    np.testing.assert_allclose(gimg, G.residual_forward(gW, 1e4)[0], atol=1e-12)
    assert gs == 0.0


@pytest.mark.parametrize("gray", [False, True])
def test_mle_vjp_matches_central_differences(gray):
    rng = np.random.default_rng(5)
    Wr = rng.standard_normal((4, 3, 8, 8))
    S = rng.uniform(50, 200, (4, 3, 8, 8))
    gK = rng.standard_normal((8, 8) if gray else (3, 8, 8))
    gW, gS = G.mle_vjp(G.mle_forward(Wr, S, gray)[1], gK)
    vW, vS = rng.standard_normal(Wr.shape), rng.standard_normal(S.shape)
    f = lambda t: float(np.sum(gK * G.mle_forward(Wr + t * vW, S + t * vS, gray)[0]))
    want = float(np.sum(gW * vW) + np.sum(gS * vS))
    assert abs((f(1e-6) - f(-1e-6)) / 2e-6 - want) <= 1e-7 * max(1.0, abs(want))


@pytest.mark.parametrize("C", [1, 3])
def test_pce_vjp_matches_central_differences_and_invariances(C):
    rng = np.random.default_rng(6)
    H, W = 32, 24
    K = rng.standard_normal((H, W)) * 0.01
    Iq = rng.uniform(40, 220, (C, H, W))
    Wq = 0.6 * K[None] * Iq + rng.standard_normal((C, H, W))
    pce, cache = G.pce_forward(K, Wq, Iq, nbhd=5)
    assert pce == pytest.approx(O.pce_match(K, O.to_gray(Wq), O.to_gray(Iq), nbhd=5).pce, rel=1e-12)
    gK, gWq = G.pce_vjp(cache, 1.0)
    vK, vW = rng.standard_normal(K.shape) * 0.01, rng.standard_normal(Wq.shape)
    f = lambda t: G.pce_forward(K + t * vK, Wq + t * vW, Iq, nbhd=5)[0]
    want = float(np.sum(gK * vK) + np.sum(gWq * vW))
    assert abs((f(1e-6) - f(-1e-6)) / 2e-6 - want) <= 1e-6 * max(1.0, abs(want))
    scale = float(np.abs(gK).sum() * np.abs(K).max() + np.abs(gWq).sum() * np.abs(Wq).max())
    assert abs(float(np.sum(gK * K))) <= 1e-9 * scale         # PCE(a K) = PCE(K)
    assert abs(float(np.sum(gWq * Wq))) <= 1e-9 * scale       # PCE(a W_q) = PCE(W_q)
    assert abs(float(np.sum(gWq))) <= 1e-9 * scale            # W_q + const


def test_sda_weighted_equal_weights_is_the_sda_mean():
    rng = np.random.default_rng(7)
    frames = rng.integers(0, 256, (13, 8, 10, 3), dtype=np.uint8)
    d = 4
    w = np.array([1.0 / min(d, 13 - (j // d) * d) for j in range(13)])
    np.testing.assert_allclose(G.sda_weighted(frames, w, d), O.sda_average(frames, d), atol=1e-12)
    gS = rng.standard_normal((4, 3, 8, 10))
    v = rng.standard_normal(13)
    f = lambda t: float(np.sum(gS * G.sda_weighted(frames, w + t * v, d)))
    assert (f(1.0) - f(-1.0)) / 2 == pytest.approx(float(np.sum(G.sda_weighted_vjp(frames, d, gS) * v)), rel=1e-12)


def test_whole_chain_gradient_matches_central_differences():
    rng = np.random.default_rng(8)
    prm = O.Params(levels=3)
    H, W, m, d = 32, 32, 12, 4
    K = rng.standard_normal((H, W)) * 0.02
    frames = np.clip(np.rint(_scene(rng, (m, H, W), 3.0) * (1 + K) + rng.standard_normal((m, H, W)) * 2),
                     0, 255).astype(np.uint8)
    q = _scene(rng, (2, 1, H, W), 3.0) * (1 + K)
    q = q + rng.standard_normal(q.shape) * 2
    w = np.full(m, 1.0 / d)
    J, gw, gs = G.objective_and_grad(frames, d, w, 3.0, q, prm, nbhd=5)
    assert J == pytest.approx(G.objective(frames, d, w, 3.0, q, prm, nbhd=5), rel=1e-12)
    v = rng.standard_normal(m) * 0.01
    fd = (G.objective(frames, d, w + 1e-6 * v, 3.0, q, prm, 5) - G.objective(frames, d, w - 1e-6 * v, 3.0, q, prm, 5)) / 2e-6
    assert fd == pytest.approx(float(gw @ v), rel=1e-5, abs=1e-6 * abs(J))
    fs = (G.objective(frames, d, w, 3.0 + 1e-6, q, prm, 5) - G.objective(frames, d, w, 3.0 - 1e-6, q, prm, 5)) / 2e-6
    assert fs == pytest.approx(gs, rel=1e-5, abs=1e-6 * abs(J))
