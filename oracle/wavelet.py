"""Daubechies filter derivation and the explicit-matrix DWT (oracle, FP64).

TEST INFRASTRUCTURE ONLY.

The paper names the denoiser only by citation (Sec. II-A and III-A point to the
wavelet filter of Mihcak et al.; Sec. IV says a wavelet denoiser was used).  The
build reads it as an
orthonormal 8-tap Daubechies wavelet (4 vanishing moments).  The lowpass filter
is derived here from Daubechies' construction rather than typed in:

  |m0(w)|^2 = cos^{2p}(w/2) P(sin^2(w/2)),   P(y) = sum_{k<p} C(p-1+k, k) y^k,

with y = (2 - z - 1/z)/4 for z on the unit circle.  z^{p-1} P(y(z)) is a
degree 2(p-1) polynomial whose roots come in reciprocal pairs; keeping the root
of each pair outside the unit circle (in the variable z, where the filter is
h(z) = sum_k h_k z^k) gives the minimum-phase factor, and

  h(z) = c ((1 + z)/2)^p prod (z - r_i),   c such that sum_k h_k = sqrt(2).
"""
from __future__ import annotations

from functools import lru_cache
from math import comb, sqrt

import numpy as np
from numpy.polynomial import polynomial as P


@lru_cache(maxsize=None)
def daubechies_lowpass(p: int = 4) -> tuple:
    """Minimum-phase Daubechies lowpass filter with p vanishing moments (2p taps)."""
    if p < 1:
        raise ValueError("p >= 1")
    # Q(z) = z^{p-1} sum_k C(p-1+k,k) y^k with y z = -(z-1)^2/4
    q = np.zeros(1)
    for k in range(p):
        term = np.array([comb(p - 1 + k, k) * (-0.25) ** k])
        for _ in range(k):
            term = P.polymul(term, [1.0, -2.0, 1.0])  # (z-1)^2 = 1 - 2z + z^2 (ascending)
        term = P.polymul(term, np.eye(1, p - k, p - 1 - k)[0])  # * z^{p-1-k}
        q = P.polyadd(q, term)
    roots = P.polyroots(q) if len(q) > 1 else np.array([])
    keep = [r for r in roots if abs(r) > 1.0]
    lfac = np.array([1.0 + 0j])
    for r in keep:
        lfac = P.polymul(lfac, [-r, 1.0])  # (z - r)
    hz = lfac
    for _ in range(p):
        hz = P.polymul(hz, [0.5, 0.5])
    hz = np.real_if_close(hz, tol=1e6).real
    hz = hz * (sqrt(2.0) / hz.sum())
    # polish to full precision with Newton steps on the defining equations
    hz = _polish(hz, p)
    return tuple(float(v) for v in hz)


def _equations(h: np.ndarray, p: int) -> np.ndarray:
    L = len(h)
    eqs = []
    for n in range(p):  # double-shift orthonormality
        s = sum(h[k] * h[k + 2 * n] for k in range(L - 2 * n))
        eqs.append(s - (1.0 if n == 0 else 0.0))
    k = np.arange(L, dtype=np.float64)
    sgn = (-1.0) ** k
    eqs.append(np.sum(h) - sqrt(2.0))
    for q in range(p):  # vanishing moments 0..p-1 of the highpass, each linear in h
        eqs.append(np.sum(sgn * k ** q * h))
    return np.array(eqs)


def _polish(h: np.ndarray, p: int, iters: int = 6) -> np.ndarray:
    h = np.array(h, dtype=np.float64)
    for _ in range(iters):
        f = _equations(h, p)
        J = np.zeros((len(f), len(h)))
        eps = 1e-7
        for j in range(len(h)):
            hp = h.copy(); hp[j] += eps
            hm = h.copy(); hm[j] -= eps
            J[:, j] = (_equations(hp, p) - _equations(hm, p)) / (2 * eps)
        step = np.linalg.lstsq(J, f, rcond=None)[0]
        h = h - step
    return h


def highpass(h) -> np.ndarray:
    """g[k] = (-1)^k h[L-1-k]."""
    h = np.asarray(h, dtype=np.float64)
    L = len(h)
    return np.array([(-1.0) ** k * h[L - 1 - k] for k in range(L)])


def dwt_matrix_1d(N: int, h) -> np.ndarray:
    """Explicit N x N matrix of one periodised analysis level on a length-N
    line: rows 0..N/2-1 give a[n], rows N/2..N-1 give d[n]."""
    h = np.asarray(h, dtype=np.float64)
    g = highpass(h)
    A = np.zeros((N, N))
    for n in range(N // 2):
        for k in range(len(h)):
            A[n, (2 * n + k) % N] += h[k]
            A[N // 2 + n, (2 * n + k) % N] += g[k]
    return A
