"""Pins of the oracle's SDA mean, MLE estimator, finalize steps and PCE
(CPU only)."""
import numpy as np
import pytest

import oracle as O
from paper_1909_04573_gb300 import synth


def test_sda_average_equals_brute_force_mean_with_ragged_group():
    rng = np.random.default_rng(0)
    fr = rng.integers(0, 256, size=(11, 9, 7, 3), dtype=np.uint8)
    out = O.sda_average(fr, 4)
    assert out.shape == (3, 3, 9, 7)
    for i, (a, b) in enumerate([(0, 4), (4, 8), (8, 11)]):
        ref = fr[a:b].astype(np.float64).mean(axis=0).transpose(2, 0, 1)
        np.testing.assert_array_equal(out[i], ref)


def test_sda_noise_variance_drops_by_d():
    # Sec. III-B: Var(psi^SDA) = sigma1^2 / d for i.i.d. noise.  Pure-noise
    # frames (mean 128, sigma 8, quantised) averaged in groups of d.
    rng = np.random.default_rng(1)
    m, d, H, W = 64, 16, 64, 64
    fr = np.clip(np.round(128 + rng.normal(0, 8, size=(m, H, W))), 0, 255).astype(np.uint8)
    sda = O.sda_average(fr, d)[:, 0]
    s1 = fr.astype(np.float64).var()
    v = sda.var(axis=(1, 2), ddof=1).mean()
    n = (m // d) * (H * W - 1)
    # chi-square with n dof: 5 sigma band on the variance ratio
    assert abs(v / (s1 / d) - 1) < 5 * np.sqrt(2.0 / n)


def test_mle_recovers_planted_fingerprint_exactly():
    # Sec. III-A: with W_i = I_i K exactly, K-hat = sum W I / sum I^2 = K.
    rng = np.random.default_rng(2)
    K = rng.normal(0, 0.005, size=(2, 16, 16))
    num = np.zeros_like(K)
    den = np.zeros_like(K)
    for _ in range(5):
        I = rng.uniform(10, 250, size=K.shape)
        O.mle_accumulate(I * K, I, num, den)
    np.testing.assert_allclose(O.fingerprint_finalize(num, den), K, atol=1e-12, rtol=0)


def test_finalize_zero_den_and_flags():
    num = np.array([[[1.0, 2.0], [3.0, 4.0]]])
    den = np.array([[[2.0, 0.0], [1.0, 8.0]]])
    np.testing.assert_array_equal(O.fingerprint_finalize(num, den), [[[0.5, 0.0], [3.0, 0.5]]])
    rng = np.random.default_rng(3)
    num3 = rng.normal(size=(3, 8, 12))
    den3 = rng.uniform(1, 2, size=(3, 8, 12))
    K = O.fingerprint_finalize(num3, den3, O.TO_GRAY | O.ZERO_MEAN)
    assert K.shape == (1, 8, 12)
    np.testing.assert_allclose(K[0].mean(axis=0), 0, atol=1e-14)
    np.testing.assert_allclose(K[0].mean(axis=1), 0, atol=1e-14)
    g = 0.299 * num3[0] / den3[0] + 0.587 * num3[1] / den3[1] + 0.114 * num3[2] / den3[2]
    g = g - g.mean(axis=0, keepdims=True)
    np.testing.assert_allclose(K[0], g - g.mean(axis=1, keepdims=True), atol=1e-14)


def test_wiener_dft_keeps_white_noise_and_removes_a_periodic_pattern():
    rng = np.random.default_rng(4)
    H, W = 64, 64
    white = rng.normal(0, 1, size=(H, W))
    out = O.wiener_dft(white)
    # a flat spectrum passes nearly unchanged
    assert np.linalg.norm(out - white) / np.linalg.norm(white) < 0.35
    yy, xx = np.mgrid[0:H, 0:W]
    pattern = 3.0 * np.cos(2 * np.pi * 8 * xx / W)  # one strong spectral peak
    out2 = O.wiener_dft(white + pattern)
    residual_pattern = np.abs(np.fft.fft2(out2))[0, 8] / np.abs(np.fft.fft2(pattern))[0, 8]
    assert residual_pattern < 0.05


def test_wiener_dft_exact_properties():
    """A constant plane has zero noise variance, so nothing passes; the
    filter is homogeneous of degree 1 (magnitudes and the noise variance
    scale together: a sigma used where sigma^2 belongs breaks this); and it
    keeps the phase of every bin it lets through."""
    np.testing.assert_allclose(O.wiener_dft(np.full((16, 24), 3.7)), 0.0, atol=1e-12)
    rng = np.random.default_rng(11)
    K = rng.normal(0, 1, size=(32, 48)) + 2.0 * np.cos(2 * np.pi * 5 * np.arange(48) / 48)[None]
    out = O.wiener_dft(K)
    np.testing.assert_allclose(O.wiener_dft(7.3 * K), 7.3 * out, rtol=1e-10, atol=1e-12)
    Fi, Fo = np.fft.fft2(K), np.fft.fft2(out)
    keep = np.abs(Fo) > 1e-9 * np.abs(Fo).max()
    assert keep.sum() > K.size // 2
    # same direction in the complex plane: Fo / Fi is real and non-negative where kept
    ratio = Fo[keep] / Fi[keep]
    np.testing.assert_allclose(ratio.imag, 0.0, atol=1e-9)
    assert (ratio.real > 0).all() and (ratio.real <= 1 + 1e-12).all()


def test_wiener_dft_equals_an_independent_route():
    """The whole DFT Wiener step computed without the oracle's code: the 2-D
    DFT as explicit matrices exp(-2 pi i k n / N), the magnitude scaled by
    1/sqrt(HW), the window means of its square by scipy's periodic box filter,
    the shrink n = M s^2 / (max(0, min_w mean_w - s^2) + s^2) with s^2 the
    plane's variance, and the inverse DFT (conjugate matrices / HW) of the
    spectrum scaled by n / M."""
    from scipy import ndimage
    rng = np.random.default_rng(12)
    H, W = 24, 40
    yy, xx = np.mgrid[0:H, 0:W]
    K = (rng.normal(0, 1, size=(H, W)) + 1.5 * np.cos(2 * np.pi * 3 * xx / W)
         + 0.8 * np.sin(2 * np.pi * (2 * yy / H + 5 * xx / W)))
    K = K - K.mean(axis=0, keepdims=True)
    K = K - K.mean(axis=1, keepdims=True)
    EH = np.exp(-2j * np.pi * np.outer(np.arange(H), np.arange(H)) / H)
    EW = np.exp(-2j * np.pi * np.outer(np.arange(W), np.arange(W)) / W)
    F = EH @ K @ EW.T
    M = np.abs(F) / np.sqrt(H * W)
    s2 = float(np.mean((K - K.mean()) ** 2))
    m = np.min([ndimage.uniform_filter(M * M, size=w, mode="wrap") for w in (3, 5, 7, 9)], axis=0)
    n = M * s2 / (np.maximum(0.0, m - s2) + s2)
    ref = np.real(EH.conj() @ (F * np.where(M > 0, n / np.where(M > 0, M, 1.0), 0.0)) @ EW.conj().T) / (H * W)
    out = O.wiener_dft(K)
    np.testing.assert_allclose(out, ref, atol=1e-11 * np.abs(K).max(), rtol=0)
    assert np.linalg.norm(out - K) > 0.05 * np.linalg.norm(K)   # the filter does something here


def _brute_correlation(X, Y):
    H, W = X.shape
    C = np.zeros((H, W))
    for sy in range(H):
        for sx in range(W):
            C[sy, sx] = np.sum(X * np.roll(np.roll(Y, -sy, axis=0), -sx, axis=1))
    return C


def test_cross_correlation_matches_brute_force():
    rng = np.random.default_rng(5)
    X, Y = rng.normal(size=(2, 12, 10))
    # C(s) = sum_x X(x) Y(x+s): a Y shifted by (3, 4) against X peaks at s=(3, 4)
    np.testing.assert_allclose(O.cross_correlation(X, Y), _brute_correlation(X, Y), atol=1e-10)
    Ys = np.roll(np.roll(X, 3, axis=0), 4, axis=1)
    C = O.cross_correlation(X, Ys)
    assert np.unravel_index(np.argmax(C), C.shape) == (3, 4)


def test_pce_matches_brute_force_definition_32x32():
    rng = np.random.default_rng(6)
    K = rng.normal(0, 0.01, size=(32, 32))
    Iq = rng.uniform(50, 200, size=(32, 32))
    Wq = K * Iq + rng.normal(0, 0.5, size=(32, 32))
    r = O.pce_match(K, Wq, Iq, nbhd=11)
    X = Wq - Wq.mean()
    Y = K * Iq - (K * Iq).mean()
    C = _brute_correlation(X, Y)
    keep = np.ones((32, 32), bool)
    for dy in range(-5, 6):
        for dx in range(-5, 6):
            keep[dy % 32, dx % 32] = False
    ref = np.sign(C[0, 0]) * C[0, 0] ** 2 / np.mean(C[keep] ** 2)
    assert abs(r.pce - ref) <= 1e-9 * abs(ref)
    assert abs(r.ncc - C[0, 0] / np.linalg.norm(X) / np.linalg.norm(Y)) < 1e-12
    assert r.peak == (0, 0)


def test_pce_and_ncc_are_odd_in_the_query_residual():
    # C -> -C when W_q -> -W_q: C(0) changes sign, the energy does not, so PCE
    # and NCC change sign with the same magnitude (an anti-correlated query is
    # a large negative PCE, not a match)
    rng = np.random.default_rng(8)
    K = rng.normal(0, 0.01, size=(32, 40))
    Iq = rng.uniform(50, 200, size=(32, 40))
    Wq = K * Iq + rng.normal(0, 0.5, size=(32, 40))
    pos, neg = O.pce_match(K, Wq, Iq), O.pce_match(K, -Wq, Iq)
    assert pos.pce > 60 and neg.pce < -60
    assert abs(neg.pce + pos.pce) <= 1e-12 * abs(pos.pce)
    assert abs(neg.ncc + pos.ncc) <= 1e-15


def test_pce_of_white_signal_with_itself_is_about_n():
    # C(0) = |X|^2 ~ N, C(s != 0) ~ N(0, N): PCE ~ N = H W
    rng = np.random.default_rng(7)
    H, W = 64, 64
    X = rng.normal(size=(H, W))
    r = O.pce_match(np.ones((H, W)), X, X)
    assert 0.85 * H * W < r.pce < 1.15 * H * W


def test_pce_of_independent_white_signals_is_order_one():
    rng = np.random.default_rng(8)
    vals = []
    for _ in range(20):
        X, Y = rng.normal(size=(2, 64, 64))
        vals.append(O.pce_match(np.ones((64, 64)), X, Y).pce)
    vals = np.abs(vals)
    assert np.max(vals) < 30 and np.mean(vals) < 3


@pytest.mark.slow
def test_planted_camera_end_to_end_small():
    # 64 grayscale 256x256 frames, SDA groups of 8 (8 denoise calls); one query
    # frame from the same camera and one from a foreign camera (Sec. IV
    # threshold 60 separates them)
    cam = synth.Camera(H=256, W=256, C=1, camera_id=7)
    fr = synth.frames(cam, 64).numpy()
    num, den = O.fingerprint_accumulate(fr, 8)
    K = O.fingerprint_finalize(num, den)[0]
    Kt = synth.k_true(cam).numpy()[0].astype(np.float64)
    assert np.corrcoef(K.ravel(), Kt.ravel())[0, 1] > 0.5
    q = synth.frames(cam, 1, stream=1).numpy()[0, :, :, 0].astype(np.float64)
    f = synth.frames(synth.foreign(cam), 1, stream=1).numpy()[0, :, :, 0].astype(np.float64)
    pos = O.pce_match(K, O.residual(q), q).pce
    neg = O.pce_match(K, O.residual(f), f).pce
    assert pos > 600 and abs(neg) < 60


@pytest.mark.slow
def test_more_groups_give_a_better_fingerprint_and_sda_costs_little_on_smooth_scenes():
    cam = synth.Camera(H=128, W=128, C=1, camera_id=9)
    fr = synth.frames(cam, 64).numpy()
    Kt = synth.k_true(cam).numpy()[0].astype(np.float64)

    def corr(m, d):
        num, den = O.fingerprint_accumulate(fr[:m], d)
        return np.corrcoef(O.fingerprint_finalize(num, den)[0].ravel(), Kt.ravel())[0, 1]

    assert corr(16, 4) < corr(64, 4)                    # more frames, better K
    # smooth scenes: the SDA estimator is close to the per-frame one (Sec. III remarks)
    assert corr(64, 4) > 0.8 * corr(64, 1)


def test_oracle_results_do_not_depend_on_the_thread_count():
    rng = np.random.default_rng(11)
    frames = rng.integers(0, 256, size=(6, 40, 56, 3), dtype=np.uint8)
    ref = O.fingerprint_accumulate(frames, 3)
    try:
        assert O.set_threads(1) == 1
        one = O.fingerprint_accumulate(frames, 3)
    finally:
        O.set_threads(None)
    np.testing.assert_array_equal(one[0], ref[0])
    np.testing.assert_array_equal(one[1], ref[1])
