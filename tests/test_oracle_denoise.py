"""Pins of the oracle's denoiser F and residual W = I - F(I) (CPU only)."""
import os

import numpy as np
import pytest
from scipy import ndimage

import oracle as O


def _rng(seed):
    return np.random.default_rng(seed)


def _scene(H, W, seed, sigma=4.0, noise=2.0):
    rng = _rng(seed)
    x = ndimage.gaussian_filter(rng.standard_normal((H, W)), sigma, mode="wrap")
    x = (x - x.mean()) / x.std() * 40 + 128
    return x + rng.normal(0, noise, size=(H, W))


def test_constant_image_has_zero_residual():
    for shape in [(16, 16), (37, 50), (64, 64)]:
        img = np.full(shape, 117.25)
        assert np.abs(O.residual(img)).max() < 1e-9


def test_sigma0_zero_gives_zero_residual():
    img = _scene(48, 64, 1)
    assert np.abs(O.residual(img, O.Params(sigma0=0.0))).max() < 1e-9


def test_large_sigma0_projects_onto_coarsest_lowpass():
    # sigma0 -> infinity: every detail is shrunk to 0, so F = IDWT(LL4 only)
    img = _scene(64, 64, 2)
    p = O.Params(sigma0=1e12)
    coeffs = O.wavedec2(img, p)
    only_ll = [coeffs[0]] + [tuple(np.zeros_like(b) for b in t) for t in coeffs[1:]]
    F = O.waverec2(only_ll, p)
    np.testing.assert_allclose(O.residual(img, p), img - F, atol=1e-9)


def test_homogeneity():
    img = _scene(64, 48, 3)
    a = 2.5
    w1 = O.residual(img, O.Params(sigma0=3.0))
    w2 = O.residual(a * img, O.Params(sigma0=3.0 * a))
    np.testing.assert_allclose(w2, a * w1, atol=1e-9)


def test_transpose_equivariance():
    img = _scene(64, 80, 4)
    np.testing.assert_allclose(O.residual(img.T), O.residual(img).T, atol=1e-9)


def test_shift_by_16_equivariance():
    img = _scene(64, 64, 5)
    shifted = np.roll(np.roll(img, 16, axis=0), -32, axis=1)
    np.testing.assert_allclose(O.residual(shifted), np.roll(np.roll(O.residual(img), 16, axis=0), -32, axis=1),
                               atol=1e-9)


def test_noise_form_equals_clean_form():
    img = _scene(40, 56, 6)
    np.testing.assert_allclose(O.residual_noise_form(img), O.residual(img), atol=1e-9)


@pytest.mark.parametrize("shape", [(16, 16), (12, 20), (5, 3)])
def test_window_means_match_library_box_filter(shape):
    # var = max(0, min_w mean_w - s0^2); the window means are periodic box means,
    # which scipy computes independently with mode='wrap'.
    c = _rng(7).standard_normal(shape) * 4
    s0 = 1.5
    _, _, var = O.shrink_subband(c, O.Params(sigma0=s0))
    means = [ndimage.uniform_filter(c * c, size=w, mode="wrap") for w in (3, 5, 7, 9)]
    ref = np.maximum(0.0, np.min(means, axis=0) - s0 * s0)
    np.testing.assert_allclose(var, ref, atol=1e-12)


def test_shrink_outputs_split_the_coefficient():
    c = _rng(8).standard_normal((16, 16)) * 5
    noise, clean, var = O.shrink_subband(c)
    np.testing.assert_allclose(noise + clean, c, atol=1e-12)
    np.testing.assert_allclose(noise, c * 9.0 / (var + 9.0), atol=1e-12)


def test_mirror_pad_repeats_the_edge():
    img = np.arange(13 * 14, dtype=np.float64).reshape(13, 14)
    p = O.pad_mirror(img, 4)
    assert p.shape == (16, 16)
    np.testing.assert_array_equal(p[13, :14], img[12])
    np.testing.assert_array_equal(p[14, :14], img[11])
    np.testing.assert_array_equal(p[15, :14], img[10])
    assert p[15, 15] == img[10, 12]
    np.testing.assert_array_equal(p[:13, 14], img[:, 13])
    np.testing.assert_array_equal(p[:13, 15], img[:, 12])
    np.testing.assert_array_equal(p[:13, :14], img)


def test_residual_of_padded_size_is_cropped():
    img = _scene(37, 50, 9)
    w = O.residual(img)
    assert w.shape == img.shape
    full = O.residual(O.pad_mirror(img, 4))
    # the padded computation is the same transform, so the crop agrees
    np.testing.assert_allclose(w, full[:37, :50], atol=1e-9)


def test_residual_is_small_on_smooth_content_and_carries_white_noise():
    rng = _rng(10)
    smooth = _scene(128, 128, 11, sigma=8.0, noise=0.0)
    noise = rng.normal(0, 2, size=(128, 128))
    w = O.residual(smooth + noise)
    # most of the white noise lands in the residual, little of the scene does
    assert np.corrcoef(w.ravel(), noise.ravel())[0, 1] > 0.8
    assert np.std(w - noise) < 1.0


# ---- the whole denoiser by an independent route ----------------------------
# The residual of a natural-looking image computed without the oracle's code:
# the taps from the published table (Daubechies 1992, Table 6.1, N = 4), the
# highpass by the quadrature-mirror relation, each periodised analysis level as
# an explicit orthogonal matrix (its rows circular shifts of the taps by 2n),
# the four levels applied to the rows and columns, numpy's symmetric padding,
# the window means by scipy's periodic box filter, the shrink
# n = c s0^2 / (max(0, min_w mean_w - s0^2) + s0^2) of every detail subband, and
# the inverse as the transposed matrices applied to (0, n) -- the noise form of
# W = I - F(I) (the residual of Sec. II-A with the denoiser's reading).

def _golden_taps():
    path = os.path.join(os.path.dirname(__file__), "golden", "daubechies_n4_lowpass.txt")
    with open(path) as f:
        return np.array([float(t) for t in (ln.strip() for ln in f) if t and not t.startswith("#")])


def _level_matrix(N, h):
    L = len(h)
    g = np.array([(-1.0) ** k * h[L - 1 - k] for k in range(L)])
    base_h, base_g = np.zeros(N), np.zeros(N)
    for k in range(L):  # taps wrap when N < L
        base_h[k % N] += h[k]
        base_g[k % N] += g[k]
    return np.vstack([np.roll(base_h, 2 * n) for n in range(N // 2)] +
                     [np.roll(base_g, 2 * n) for n in range(N // 2)])


def _residual_by_matrices(img, s0=3.0, levels=4, windows=(3, 5, 7, 9)):
    H, W = img.shape
    step = 2 ** levels
    Hp, Wp = -(-H // step) * step, -(-W // step) * step
    x = np.pad(img, ((0, Hp - H), (0, Wp - W)), mode="symmetric")
    h = _golden_taps()
    mats, noise = [], []
    for lv in range(levels):
        R, C = Hp >> lv, Wp >> lv
        Ar, Ac = _level_matrix(R, h), _level_matrix(C, h)
        y = Ar @ x @ Ac.T              # quadrants: [lo-lo, lo-hi; hi-lo, hi-hi]
        r, c = R // 2, C // 2
        n = np.zeros_like(y)
        for sl in ((slice(0, r), slice(c, C)), (slice(r, R), slice(0, c)), (slice(r, R), slice(c, C))):
            d = y[sl]
            m = np.min([ndimage.uniform_filter(d * d, size=w, mode="wrap") for w in windows], axis=0)
            n[sl] = d * s0 * s0 / (np.maximum(0.0, m - s0 * s0) + s0 * s0)
        mats.append((Ar, Ac))
        noise.append(n)
        x = y[:r, :c]
    z = np.zeros((Hp >> levels, Wp >> levels))   # the noise form keeps no lowpass
    for lv in reversed(range(levels)):
        Ar, Ac = mats[lv]
        n = noise[lv]
        r, c = z.shape
        n[:r, :c] = z
        z = Ar.T @ n @ Ac
    return z[:H, :W]


@pytest.mark.parametrize("shape,seed", [((37, 50), 21), ((64, 96), 22), ((80, 48), 23)])
def test_residual_equals_the_matrix_route(shape, seed):
    img = _scene(*shape, seed)
    ref = _residual_by_matrices(img)
    got = O.residual(img)
    # the table's 12 printed decimals bound the agreement
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(img).max()
    assert np.abs(ref).max() > 0.5       # a non-trivial residual


def test_matrix_route_with_other_parameters():
    img = _scene(48, 64, 24, noise=5.0)
    for s0, wins in ((1.0, (3, 5, 7, 9)), (5.0, (3,)), (3.0, (5, 9))):
        ref = _residual_by_matrices(img, s0=s0, windows=wins)
        got = O.residual(img, O.Params(sigma0=s0, windows=wins))
        assert np.abs(got - ref).max() <= 1e-8 * np.abs(img).max(), (s0, wins)
