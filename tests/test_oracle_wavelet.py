"""Pins of the oracle's wavelet transform against textbook values, closed forms
and the mathematics of orthonormal periodised filter banks (CPU only)."""
import os
from math import sqrt

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "daubechies_n4_lowpass.txt")


def _golden_table():
    vals = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                vals.append(float(line))
    return np.array(vals)


def test_filter_matches_textbook_table():
    # Daubechies, Ten Lectures on Wavelets, Table 6.1, N = 4 (12 printed decimals)
    h = np.array(O.daubechies_lowpass(4))
    np.testing.assert_allclose(h, _golden_table(), atol=6e-13, rtol=0)


def test_d4_closed_form():
    # N = 2: h = ((1+s3), (3+s3), (3-s3), (1-s3)) / (4 sqrt 2), s3 = sqrt 3
    s3 = sqrt(3.0)
    ref = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4 * sqrt(2.0))
    np.testing.assert_allclose(O.daubechies_lowpass(2), ref, atol=1e-15)
    np.testing.assert_allclose(O.daubechies_lowpass(1), [1 / sqrt(2.0)] * 2, atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_filter_identities(p):
    h = np.array(O.daubechies_lowpass(p))
    L = len(h)
    assert L == 2 * p
    assert abs(h.sum() - sqrt(2.0)) < 1e-14
    for n in range(p):
        s = sum(h[k] * h[k + 2 * n] for k in range(L - 2 * n))
        assert abs(s - (1.0 if n == 0 else 0.0)) < 1e-14
    k = np.arange(L, dtype=np.float64)
    for q in range(p):  # vanishing moments of the highpass, including q = 0
        assert abs(np.sum((-1.0) ** k * k ** q * h)) < 1e-12 * max(1.0, (L - 1) ** q)
    # minimum phase: the roots of sum_k h_k z^k lie outside the unit circle
    roots = np.roots(h[::-1])
    finite = roots[np.abs(roots + 1) > 1e-3]  # drop the p-fold root at z = -1
    assert np.all(np.abs(finite) > 1.0)


def _full_dwt_matrix(N, levels):
    """Matrix of the full levels-deep 2-D DWT on N x N images, built by pushing
    unit images through the oracle (so it pins the C code)."""
    cols = []
    for i in range(N * N):
        e = np.zeros(N * N)
        e[i] = 1.0
        coeffs = O.wavedec2(e.reshape(N, N), O.Params(levels=levels))
        flat = [coeffs[0].ravel()] + [b.ravel() for trip in coeffs[1:] for b in trip]
        cols.append(np.concatenate(flat))
    return np.array(cols).T


def test_explicit_matrix_parseval_16x16():
    A = _full_dwt_matrix(16, 4)
    assert A.shape == (256, 256)
    np.testing.assert_allclose(A.T @ A, np.eye(256), atol=1e-12)
    np.testing.assert_allclose(A @ A.T, np.eye(256), atol=1e-12)


def test_separable_matrix_matches_c_code():
    # one level of the 2-D transform equals the 1-D matrix applied to rows,
    # then to columns, with the subbands in the documented places
    rng = np.random.default_rng(1)
    R, Cc = 16, 24
    x = rng.standard_normal((R, Cc))
    h = O.DEFAULT.h
    Ar, Ac = O.dwt_matrix_1d(Cc, h), O.dwt_matrix_1d(R, h)
    rows = x @ Ar.T                     # per row: [lo | hi]
    full = Ac @ rows                    # per column: [lo ; hi]
    LL, LH, HL, HH = O.dwt2_level(x)
    np.testing.assert_allclose(LL, full[:R // 2, :Cc // 2], atol=1e-12)
    np.testing.assert_allclose(LH, full[R // 2:, :Cc // 2], atol=1e-12)   # row-low, col-high
    np.testing.assert_allclose(HL, full[:R // 2, Cc // 2:], atol=1e-12)   # row-high, col-low
    np.testing.assert_allclose(HH, full[R // 2:, Cc // 2:], atol=1e-12)


@pytest.mark.parametrize("shape", [(16, 16), (32, 48), (64, 64), (128, 80), (256, 256)])
def test_perfect_reconstruction(shape):
    rng = np.random.default_rng(shape[0] * 1000 + shape[1])
    x = rng.uniform(0, 255, size=shape)
    coeffs = O.wavedec2(x)
    assert np.abs(O.waverec2(coeffs) - x).max() <= 1e-10
    energy = coeffs[0].ravel() @ coeffs[0].ravel() + sum((b * b).sum() for t in coeffs[1:] for b in t)
    assert abs(energy - (x * x).sum()) <= 1e-10 * (x * x).sum()


def test_polynomials_are_annihilated_away_from_the_wrap():
    # 4 vanishing moments: a cubic along x leaves every row-high coefficient 0
    # except where the filter wraps around the periodic boundary.
    N = 64
    xs = np.arange(N, dtype=np.float64)
    img = np.tile(0.01 * xs ** 3 - 0.5 * xs ** 2 + 3 * xs + 7, (N, 1))  # varies along columns index
    LL, LH, HL, HH = O.dwt2_level(img)
    interior = slice(0, N // 2 - 4)  # taps 2n..2n+7 stay inside [0, N)
    assert np.abs(HL[:, interior]).max() < 1e-8
    assert np.abs(HH[:, interior]).max() < 1e-8
    assert np.abs(LH).max() < 1e-8  # constant along rows direction -> col-high is 0
    assert np.abs(HL[:, N // 2 - 1]).max() > 1.0  # the wrap is visible


def test_subband_naming_vertical_and_horizontal_stripes():
    N = 32
    stripes_x = np.tile((-1.0) ** np.arange(N), (N, 1))     # alternates along x (columns)
    LL, LH, HL, HH = O.dwt2_level(stripes_x)
    assert np.abs(HL).max() > 1.0 and np.abs(LH).max() < 1e-12 and np.abs(HH).max() < 1e-12
    LL, LH, HL, HH = O.dwt2_level(stripes_x.T)               # alternates along y (rows)
    assert np.abs(LH).max() > 1.0 and np.abs(HL).max() < 1e-12 and np.abs(HH).max() < 1e-12
