"""FP64 oracle of the SDA fingerprint pipeline (numpy + the plain-C core).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU legs of bench.py, never by the CUDA product path.

Steps, in the paper's order:
  sda_average            Sec. III-B, definition of I_i^SDA (mean of d frames)
  residual               Sec. II-A, W = I - F(I); F = the wavelet denoiser
  fingerprint_accumulate Sec. III-A equation for K-hat / Sec. III-B K-hat^SDA:
                         num = sum W.I, den = sum I^2
  fingerprint_finalize   K = num/den (Sec. III-A); zero-mean, DFT-domain Wiener
                         and grey conversion are literature steps the paper
                         does not define (optional flags)
  pce_match              Sec. IV: PCE with threshold 60 (definition by
                         citation only; the reading used is stated below)

Readings where the paper is silent (all listed in the design notes): 8-tap
Daubechies, orthonormal, periodised DWT, 4 levels, windows 3/5/7/9 with
periodic wrap, sigma0 = 3, mirror padding to multiples of 2^levels, per-channel
residual and MLE, mean over the actual frame count for a ragged last group.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import native
from .wavelet import daubechies_lowpass

ZERO_MEAN = 1
WIENER_DFT = 2
TO_GRAY = 4

GRAY_WEIGHTS = (0.299, 0.587, 0.114)


@dataclass(frozen=True)
class Params:
    levels: int = 4
    sigma0: float = 3.0
    windows: tuple = (3, 5, 7, 9)
    vanishing_moments: int = 4  # 8 taps

    @property
    def h(self) -> np.ndarray:
        return np.array(daubechies_lowpass(self.vanishing_moments), dtype=np.float64)


DEFAULT = Params()


def padded_size(n: int, levels: int) -> int:
    m = 1 << levels
    return (n + m - 1) // m * m


# --------------------------------------------------------------------------
# SDA frames (Sec. III-B)
# --------------------------------------------------------------------------
def sda_average(frames: np.ndarray, d: int) -> np.ndarray:
    """frames uint8 [m, H, W, C] (or [m, H, W]) -> float64 [g, C, H, W].

    Group i holds frames i*d .. min((i+1)*d, m) - 1; its SDA frame is their mean.
    """
    if frames.ndim == 3:
        frames = frames[..., None]
    frames = np.ascontiguousarray(frames, dtype=np.uint8)
    m, H, W, C = frames.shape
    g = (m + d - 1) // d
    out = np.zeros((g, C, H, W), dtype=np.float64)
    rc = native.lib().orc_sda_average(frames.ctypes.data, m, H, W, C, H * W * C, W * C, d,
                                      native.dptr(out))
    native.check(rc, "sda_average")
    return out


# --------------------------------------------------------------------------
# DWT building blocks (exposed for the pins)
# --------------------------------------------------------------------------
def dwt2_level(x: np.ndarray, params: Params = DEFAULT):
    x = np.ascontiguousarray(x, dtype=np.float64)
    R, Cc = x.shape
    outs = [np.zeros((R // 2, Cc // 2)) for _ in range(4)]
    h = params.h
    rc = native.lib().orc_dwt2_level(native.dptr(x), R, Cc, native.dptr(h), len(h),
                                     *[native.dptr(o) for o in outs])
    native.check(rc, "dwt2_level")
    return tuple(outs)  # LL, LH, HL, HH


def idwt2_level(LL, LH, HL, HH, params: Params = DEFAULT) -> np.ndarray:
    bands = [np.ascontiguousarray(b, dtype=np.float64) for b in (LL, LH, HL, HH)]
    R, Cc = 2 * bands[0].shape[0], 2 * bands[0].shape[1]
    x = np.zeros((R, Cc))
    h = params.h
    rc = native.lib().orc_idwt2_level(*[native.dptr(b) for b in bands], R, Cc, native.dptr(h), len(h),
                                      native.dptr(x))
    native.check(rc, "idwt2_level")
    return x


def wavedec2(x: np.ndarray, params: Params = DEFAULT):
    """Full pyramid: [LL_L, (LH_L, HL_L, HH_L), ..., (LH_1, HL_1, HH_1)]."""
    details = []
    ll = np.ascontiguousarray(x, dtype=np.float64)
    for _ in range(params.levels):
        ll, lh, hl, hh = dwt2_level(ll, params)
        details.append((lh, hl, hh))
    return [ll] + details[::-1]


def waverec2(coeffs, params: Params = DEFAULT) -> np.ndarray:
    ll = coeffs[0]
    for lh, hl, hh in coeffs[1:]:
        ll = idwt2_level(ll, lh, hl, hh, params)
    return ll


def shrink_subband(c: np.ndarray, params: Params = DEFAULT, sigma0: float | None = None):
    """Local-variance Wiener shrink of one subband -> (noise, clean, var)."""
    c = np.ascontiguousarray(c, dtype=np.float64)
    R, Cc = c.shape
    noise, clean, var = np.zeros_like(c), np.zeros_like(c), np.zeros_like(c)
    win = np.array(params.windows, dtype=np.int32)
    s0 = params.sigma0 if sigma0 is None else sigma0
    rc = native.lib().orc_shrink_subband(native.dptr(c), R, Cc, float(s0), native.iptr(win), len(win),
                                         native.dptr(noise), native.dptr(clean), native.dptr(var))
    native.check(rc, "shrink_subband")
    return noise, clean, var


def pad_mirror(img: np.ndarray, levels: int) -> np.ndarray:
    img = np.ascontiguousarray(img, dtype=np.float64)
    H, W = img.shape
    Hp, Wp = padded_size(H, levels), padded_size(W, levels)
    out = np.zeros((Hp, Wp))
    native.check(native.lib().orc_pad_mirror(native.dptr(img), H, W, Hp, Wp, native.dptr(out)), "pad")
    return out


def denoise_plane(xp: np.ndarray, params: Params = DEFAULT):
    """Padded plane -> (F, Wn): F = IDWT(LL_L, clean details) and
    Wn = IDWT(0, noise details)."""
    xp = np.ascontiguousarray(xp, dtype=np.float64)
    Hp, Wp = xp.shape
    F, Wn = np.zeros_like(xp), np.zeros_like(xp)
    h = params.h
    win = np.array(params.windows, dtype=np.int32)
    rc = native.lib().orc_denoise_plane(native.dptr(xp), Hp, Wp, params.levels, native.dptr(h), len(h),
                                        float(params.sigma0), native.iptr(win), len(win),
                                        native.dptr(F), native.dptr(Wn))
    native.check(rc, "denoise_plane")
    return F, Wn


# --------------------------------------------------------------------------
# Residual W = I - F(I)  (Sec. II-A)
# --------------------------------------------------------------------------
def residual(img: np.ndarray, params: Params = DEFAULT) -> np.ndarray:
    """img float [C, H, W] or [H, W] (0..255 units) -> W of the same shape."""
    img = np.asarray(img, dtype=np.float64)
    if img.ndim == 2:
        return residual(img[None], params)[0]
    C, H, W = img.shape
    out = np.zeros((C, H, W))
    h = params.h
    win = np.array(params.windows, dtype=np.int32)
    for c in range(C):
        plane = np.ascontiguousarray(img[c])
        res = np.zeros((H, W))
        rc = native.lib().orc_residual_plane(native.dptr(plane), H, W, params.levels, native.dptr(h),
                                             len(h), float(params.sigma0), native.iptr(win), len(win),
                                             native.dptr(res))
        native.check(rc, "residual_plane")
        out[c] = res
    return out


def residual_noise_form(img: np.ndarray, params: Params = DEFAULT) -> np.ndarray:
    """The same residual computed as IDWT(0, noise details) (linearity), cropped."""
    img = np.asarray(img, dtype=np.float64)
    if img.ndim == 2:
        return residual_noise_form(img[None], params)[0]
    C, H, W = img.shape
    out = np.zeros((C, H, W))
    for c in range(C):
        _, Wn = denoise_plane(pad_mirror(img[c], params.levels), params)
        out[c] = Wn[:H, :W]
    return out


# --------------------------------------------------------------------------
# MLE fingerprint (Sec. III-A, Sec. III-B)
# --------------------------------------------------------------------------
def fingerprint_accumulate(frames: np.ndarray, d: int, params: Params = DEFAULT,
                           num: np.ndarray | None = None, den: np.ndarray | None = None,
                           group_range: tuple | None = None):
    """uint8 frames [m, H, W, C] -> (num, den) float64 [C, H, W].

    num += sum_i W_i^SDA . I_i^SDA and den += sum_i (I_i^SDA)^2 over the SDA
    frames of groups of d (d = 1 is the conventional per-frame estimator).
    group_range=(i0, i1) restricts the sum to those groups (sampling).
    """
    if frames.ndim == 3:
        frames = frames[..., None]
    m, H, W, C = frames.shape
    if num is None:
        num = np.zeros((C, H, W))
    if den is None:
        den = np.zeros((C, H, W))
    g = (m + d - 1) // d
    i0, i1 = group_range if group_range is not None else (0, g)
    for i in range(i0, i1):
        sub = frames[i * d: min((i + 1) * d, m)]
        I = sda_average(sub, len(sub))[0]
        Wr = residual(I, params)
        mle_accumulate(Wr, I, num, den)
    return num, den


def mle_accumulate(Wr: np.ndarray, I: np.ndarray, num: np.ndarray, den: np.ndarray) -> None:
    """num += W.I and den += I.I elementwise (in place), the sums of the MLE
    estimator K-hat = sum W_i I_i / sum I_i^2 (Sec. III-A)."""
    Wr = np.ascontiguousarray(Wr, dtype=np.float64)
    I = np.ascontiguousarray(I, dtype=np.float64)
    assert Wr.shape == I.shape == num.shape == den.shape
    nc = np.ascontiguousarray(num)
    dc = np.ascontiguousarray(den)
    native.lib().orc_mle_accumulate(native.dptr(Wr), native.dptr(I), I.size, native.dptr(nc), native.dptr(dc))
    num[...] = nc
    den[...] = dc


def to_gray(x: np.ndarray) -> np.ndarray:
    """[3, H, W] -> [H, W] with the 0.299/0.587/0.114 weights; [1,H,W] -> [H,W]."""
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 2:
        return x
    if x.shape[0] == 1:
        return x[0].copy()
    return GRAY_WEIGHTS[0] * x[0] + GRAY_WEIGHTS[1] * x[1] + GRAY_WEIGHTS[2] * x[2]


def zero_mean(K: np.ndarray) -> np.ndarray:
    """Subtract each column's mean, then each row's mean (one plane)."""
    K = np.array(K, dtype=np.float64)
    K = K - K.mean(axis=0, keepdims=True)
    K = K - K.mean(axis=1, keepdims=True)
    return K


def wiener_dft(K: np.ndarray, params: Params = DEFAULT) -> np.ndarray:
    """DFT-domain Wiener filter of one plane: the magnitude |DFT(K)|/sqrt(N)
    goes through the same local-variance shrink (noise form) with noise
    variance var(K); the phase is kept; real part of the inverse DFT."""
    K = np.asarray(K, dtype=np.float64)
    N = K.size
    F = np.fft.fft2(K)
    M = np.abs(F) / np.sqrt(N)
    sig2 = float(np.var(K))
    noiseM, _, _ = shrink_subband(M, params, sigma0=np.sqrt(sig2))
    ratio = np.where(M > 0, noiseM / np.where(M > 0, M, 1.0), 0.0)
    return np.real(np.fft.ifft2(F * ratio))


def fingerprint_finalize(num: np.ndarray, den: np.ndarray, flags: int = 0,
                         params: Params = DEFAULT) -> np.ndarray:
    """K = num/den (0 where den == 0), then optional TO_GRAY, ZERO_MEAN,
    WIENER_DFT, applied in that order.  Returns [C, H, W] or [1, H, W]."""
    num = np.asarray(num, dtype=np.float64)
    den = np.asarray(den, dtype=np.float64)
    K = np.where(den != 0, num / np.where(den != 0, den, 1.0), 0.0)
    if flags & TO_GRAY:
        K = to_gray(K)[None]
    if flags & ZERO_MEAN:
        K = np.stack([zero_mean(k) for k in K])
    if flags & WIENER_DFT:
        K = np.stack([wiener_dft(k, params) for k in K])
    return K


# --------------------------------------------------------------------------
# PCE (Sec. IV; definition by citation only)
# --------------------------------------------------------------------------
@dataclass
class PCEResult:
    pce: float
    ncc: float
    peak: tuple = field(default=(0, 0))  # (row shift, col shift) of max C
    c0: float = 0.0
    energy: float = 0.0


def cross_correlation(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """C(s) = sum_x X(x) Y(x + s), circular, s = (row, col)."""
    return np.real(np.fft.ifft2(np.conj(np.fft.fft2(X)) * np.fft.fft2(Y)))


def pce_match(K: np.ndarray, Wq: np.ndarray, Iq: np.ndarray, nbhd: int = 11) -> PCEResult:
    """Planes [H, W] (grey or one channel): X = W_q, Y = K.I_q, both made
    zero-mean; C = circular cross-correlation; peak taken at zero shift;
    PCE = sign(C0) C0^2 / mean over s outside the nbhd x nbhd block centred at
    zero shift (wrapped) of C(s)^2; NCC = C0 / (|X| |Y|)."""
    K, Wq, Iq = (np.asarray(a, dtype=np.float64) for a in (K, Wq, Iq))
    X = Wq - Wq.mean()
    Y = K * Iq
    Y = Y - Y.mean()
    C = cross_correlation(X, Y)
    H, W = C.shape
    r = nbhd // 2
    mask = np.ones((H, W), dtype=bool)
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            mask[dy % H, dx % W] = False
    c0 = float(C[0, 0])
    energy = float(np.mean(C[mask] ** 2))
    pce = np.sign(c0) * c0 * c0 / energy if energy > 0 else 0.0
    nx, ny = np.linalg.norm(X), np.linalg.norm(Y)
    ncc = c0 / (nx * ny) if nx > 0 and ny > 0 else 0.0
    pk = np.unravel_index(int(np.argmax(C)), C.shape)
    return PCEResult(pce=float(pce), ncc=float(ncc), peak=(int(pk[0]), int(pk[1])), c0=c0, energy=energy)
