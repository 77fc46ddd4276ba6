"""FP64 adjoint (vector-Jacobian products) of the differentiable chain.

TEST INFRASTRUCTURE ONLY: imported by tests/ and the CPU legs of bench.py,
never by the CUDA product path.

The chain, for one camera (all steps of the extraction method, with the SDA
weights made free parameters):
  S_i = sum_{j in group i} w_j I_j      Sec. III-B (w_j = 1/d gives the SDA frame)
  W_i = residual(S_i; sigma0)           Sec. II-A / III-A, noise form of the
                                        wavelet denoiser (IDWT of the shrunk
                                        detail coefficients' noise part)
  K   = sum_i W_i S_i / sum_i S_i^2     Sec. III-A (MLE), grey for C = 3
  PCE of each query (W_q = residual(I_q; sigma0), I_q) against K   Sec. IV
Every function below restates one step's forward in the order of the method
and its exact derivative; the DWT levels are the oracle's own dwt2_level /
idwt2_level, whose orthonormality (the transpose of one is the other) is pinned
by the wavelet tests.  The derivative is taken away from ties between window
means (the argmin window is then locally constant) and away from
min-mean == sigma0^2 (the kink of max(0, .)).
"""
from __future__ import annotations

import numpy as np

from . import pipeline as P


# --------------------------------------------------------------------------
# weighted SDA frames (Sec. III-B with free per-frame weights)
# --------------------------------------------------------------------------
def sda_weighted(frames: np.ndarray, w: np.ndarray, d: int) -> np.ndarray:
    """uint8 frames [m, H, W, C] (or [m, H, W]), weights [m] -> S [g, C, H, W]:
    S_i = sum over frames j of group i (frames i*d .. min((i+1)d, m) - 1) of w_j I_j."""
    if frames.ndim == 3:
        frames = frames[..., None]
    m, H, W, C = frames.shape
    g = (m + d - 1) // d
    S = np.zeros((g, C, H, W))
    for j in range(m):
        S[j // d] += float(w[j]) * np.transpose(frames[j], (2, 0, 1)).astype(np.float64)
    return S


def sda_weighted_vjp(frames: np.ndarray, d: int, gS: np.ndarray) -> np.ndarray:
    """d<gS, S>/dw_j = <gS_{group(j)}, I_j>."""
    if frames.ndim == 3:
        frames = frames[..., None]
    m = frames.shape[0]
    return np.array([float(np.sum(gS[j // d] * np.transpose(frames[j], (2, 0, 1)).astype(np.float64)))
                     for j in range(m)])


# --------------------------------------------------------------------------
# local-variance Wiener shrink, noise part (denoiser of Sec. III-A / IV)
# --------------------------------------------------------------------------
def _box_sum(a: np.ndarray, w: int) -> np.ndarray:
    """Periodic w x w box sum centred on each sample."""
    r = w // 2
    s = np.zeros_like(a)
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            s += np.roll(a, (-dy, -dx), axis=(0, 1))
    return s


def shrink_forward(c: np.ndarray, sigma0: float, windows=(3, 5, 7, 9)):
    """noise = c s2 / (max(0, m - s2) + s2), m = min over windows of the
    window mean of c^2 (periodic).  Returns (noise, cache)."""
    s2 = sigma0 * sigma0
    means = np.stack([_box_sum(c * c, w) / (w * w) for w in windows])
    k = np.argmin(means, axis=0)            # first window on ties
    m = np.min(means, axis=0)
    den = np.maximum(0.0, m - s2) + s2
    noise = np.where(den > 0, c * s2 / np.where(den > 0, den, 1.0), 0.0)
    return noise, (c, m, k, den, sigma0, tuple(windows))


def shrink_vjp(cache, gn: np.ndarray):
    """-> (g_c, g_sigma0).  Where m > s2: noise = c s2 / m, so
    d/dc (direct) = s2/m, d/dm = -c s2 / m^2, d/ds2 = c/m; elsewhere noise = c
    (s2 > 0) and only the direct term is left.  m depends on c through the
    argmin window's mean: dm(p)/dc(q) = 2 c(q) / w^2 for q in p's window."""
    c, m, k, den, sigma0, windows = cache
    s2 = sigma0 * sigma0
    active = m > s2
    mm = np.where(active, m, 1.0)
    gc = gn * np.where(den > 0, s2 / np.where(den > 0, den, 1.0), 0.0)
    gm = np.where(active, -gn * c * s2 / (mm * mm), 0.0)
    for i, w in enumerate(windows):
        a = np.where(k == i, gm, 0.0) / (w * w)
        gc = gc + 2.0 * c * _box_sum(a, w)
    g_s2 = float(np.sum(np.where(active, gn * c / mm, 0.0)))
    return gc, 2.0 * sigma0 * g_s2


# --------------------------------------------------------------------------
# residual W = IDWT(0, noise(details(pad(S))))[:H, :W]   (Sec. II-A)
# --------------------------------------------------------------------------
def _mirror_index(n: int, npad: int) -> np.ndarray:
    i = np.arange(npad)
    return np.where(i < n, i, 2 * n - 1 - i)


def residual_forward(img: np.ndarray, sigma0: float, params: P.Params = P.DEFAULT):
    """img [C, H, W] -> (W [C, H, W], cache).  Same residual as
    pipeline.residual_noise_form (mirror pad, periodised orthonormal DWT)."""
    img = np.asarray(img, dtype=np.float64)
    C, H, W = img.shape
    L = params.levels
    out = np.zeros_like(img)
    caches = []
    for ch in range(C):
        ll = P.pad_mirror(img[ch], L)
        lv = []
        for _ in range(L):
            ll, lh, hl, hh = P.dwt2_level(ll, params)
            lv.append([shrink_forward(b, sigma0, params.windows) for b in (lh, hl, hh)])
        r = np.zeros_like(ll)  # LL_L of the noise part is 0
        for l in range(L - 1, -1, -1):
            r = P.idwt2_level(r, *(lv[l][b][0] for b in range(3)), params)
        out[ch] = r[:H, :W]
        caches.append(lv)
    return out, (caches, H, W, sigma0, params)


def residual_vjp(cache, gW: np.ndarray):
    """-> (g_img [C, H, W], g_sigma0).  Transposes, in reverse order: crop
    (zero-extend), IDWT levels (DWT levels), shrink, DWT levels (IDWT levels),
    mirror pad (fold the padded samples back onto their sources)."""
    caches, H, W, sigma0, params = cache
    L = params.levels
    Hp, Wp = P.padded_size(H, L), P.padded_size(W, L)
    ri, ci = _mirror_index(H, Hp), _mirror_index(W, Wp)
    g_img = np.zeros((len(caches), H, W))
    g_sigma = 0.0
    for ch, lv in enumerate(caches):
        g = np.zeros((Hp, Wp))
        g[:H, :W] = gW[ch]
        gn = []
        for _ in range(L):                     # adjoint of the synthesis chain
            g, glh, ghl, ghh = P.dwt2_level(g, params)
            gn.append((glh, ghl, ghh))
        gc = []
        for l in range(L):
            t = []
            for b in range(3):
                gcb, gs = shrink_vjp(lv[l][b][1], gn[l][b])
                t.append(gcb)
                g_sigma += gs
            gc.append(t)
        gll = np.zeros((Hp >> L, Wp >> L))      # the residual does not use LL_L
        for l in range(L - 1, -1, -1):          # adjoint of the analysis chain
            gll = P.idwt2_level(gll, *gc[l], params)
        fold = np.zeros((H, W))
        np.add.at(fold, (ri[:, None], ci[None, :]), gll)
        g_img[ch] = fold
    return g_img, g_sigma


# --------------------------------------------------------------------------
# MLE fingerprint K = sum W S / sum S^2   (Sec. III-A)
# --------------------------------------------------------------------------
def mle_forward(Wr: np.ndarray, S: np.ndarray, gray: bool = False):
    """Wr, S [n, C, H, W] -> K [C, H, W] (or [H, W] grey when gray), cache."""
    num = np.sum(Wr * S, axis=0)
    den = np.sum(S * S, axis=0)
    K = np.where(den != 0, num / np.where(den != 0, den, 1.0), 0.0)
    Kout = P.to_gray(K) if gray else K
    return Kout, (Wr, S, num, den, gray)


def mle_vjp(cache, gK: np.ndarray):
    """-> (g_Wr, g_S)."""
    Wr, S, num, den, gray = cache
    C = S.shape[1]
    if gray:
        wts = P.GRAY_WEIGHTS if C == 3 else (1.0,)
        gK = np.stack([wts[c] * gK for c in range(C)])
    ok = den != 0
    dd = np.where(ok, den, 1.0)
    g_num = np.where(ok, gK / dd, 0.0)
    g_den = np.where(ok, -gK * num / (dd * dd), 0.0)
    return g_num[None] * S, g_num[None] * Wr + 2.0 * g_den[None] * S


# --------------------------------------------------------------------------
# PCE against K (Sec. IV; same reading as pipeline.pce_match)
# --------------------------------------------------------------------------
def pce_forward(K: np.ndarray, Wq: np.ndarray, Iq: np.ndarray, nbhd: int = 11):
    """K [H, W]; Wq, Iq [C, H, W] (or [H, W]) -> (pce, cache)."""
    Wq = np.asarray(Wq, dtype=np.float64)
    Iq = np.asarray(Iq, dtype=np.float64)
    C = 1 if Wq.ndim == 2 else Wq.shape[0]
    Xg, Ig = P.to_gray(Wq), P.to_gray(Iq)
    X = Xg - Xg.mean()
    Y = K * Ig
    Y = Y - Y.mean()
    Cr = P.cross_correlation(X, Y)
    H, W = Cr.shape
    r = nbhd // 2
    mask = np.ones((H, W), dtype=bool)
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            mask[dy % H, dx % W] = False
    c0 = float(Cr[0, 0])
    E = float(np.sum(Cr[mask] ** 2))
    O = int(mask.sum())
    pce = np.sign(c0) * c0 * c0 * O / E if E > 0 else 0.0
    return float(pce), (X, Y, Cr, mask, c0, E, O, pce, Ig, C, Wq.ndim)


def pce_vjp(cache, g: float = 1.0):
    """-> (g_K [H, W], g_Wq like Wq).  With G(s) = dPCE/dC(s):
    G(0) = 2|C0| O / E, G(s) = -2 PCE C(s) / E outside the neighbourhood,
    dPCE/dX(x) = sum_s G(s) Y(x+s) (a correlation of G with Y) and
    dPCE/dY(y) = sum_s G(s) X(y-s) (a convolution of G with X); the mean
    removals and the grey weights are then transposed."""
    X, Y, Cr, mask, c0, E, O, pce, Ig, C, nd = cache
    G = np.zeros_like(Cr)
    if E > 0:
        G[mask] = -2.0 * pce * Cr[mask] / E
        G[0, 0] = 2.0 * abs(c0) * O / E
    G *= g
    gXc = P.cross_correlation(G, Y)
    gYc = np.real(np.fft.ifft2(np.fft.fft2(X) * np.fft.fft2(G)))
    gX = gXc - gXc.mean()
    gY = gYc - gYc.mean()
    gK = gY * Ig
    if nd == 2:
        gWq = gX
    else:
        wts = P.GRAY_WEIGHTS if C == 3 else (1.0,)
        gWq = np.stack([wts[c] * gX for c in range(C)])
    return gK, gWq


# --------------------------------------------------------------------------
# the whole chain: mean PCE of the queries against the camera's fingerprint
# --------------------------------------------------------------------------
def objective(frames, d, w, sigma0, qimgs, params: P.Params = P.DEFAULT, nbhd: int = 11):
    """frames uint8 [m, H, W(, C)], weights [m], qimgs float [nq, C, H, W] ->
    mean over queries of PCE(K, residual(q), q)."""
    S = sda_weighted(frames, w, d)
    Wr = np.stack([residual_forward(s, sigma0, params)[0] for s in S])
    K, _ = mle_forward(Wr, S, gray=True)
    vals = [pce_forward(K, residual_forward(q, sigma0, params)[0], q, nbhd)[0] for q in qimgs]
    return float(np.mean(vals))


def objective_and_grad(frames, d, w, sigma0, qimgs, params: P.Params = P.DEFAULT, nbhd: int = 11):
    """-> (J, g_w [m], g_sigma0)."""
    S = sda_weighted(frames, w, d)
    res = [residual_forward(s, sigma0, params) for s in S]
    Wr = np.stack([r[0] for r in res])
    K, mc = mle_forward(Wr, S, gray=True)
    nq = len(qimgs)
    gK = np.zeros_like(K)
    g_sigma = 0.0
    vals = []
    for q in qimgs:
        Wq, qc = residual_forward(q, sigma0, params)
        v, pc = pce_forward(K, Wq, q, nbhd)
        vals.append(v)
        gk, gwq = pce_vjp(pc, 1.0 / nq)
        gK += gk
        _, gs = residual_vjp(qc, gwq)
        g_sigma += gs
    gWr, gS = mle_vjp(mc, gK)
    for i, (_, rc) in enumerate(res):
        gi, gs = residual_vjp(rc, gWr[i])
        gS[i] += gi
        g_sigma += gs
    return float(np.mean(vals)), sda_weighted_vjp(frames, d, gS), g_sigma
