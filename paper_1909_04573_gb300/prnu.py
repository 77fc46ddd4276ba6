"""Thin ctypes binding of libprnu (include/prnu.h): same names, argument
marshalling only.  Every step of the path runs in the library's CUDA kernels;
there is no CPU fallback, and loading fails loudly when libprnu.so is missing.

The torch-level helpers at the bottom only turn tensors into pointers, sizes,
strides and the current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libprnu.so")

PRNU_OK, PRNU_EINVAL, PRNU_ENOSPC, PRNU_ECUDA, PRNU_ETIMEOUT, PRNU_EUNSUPPORTED, PRNU_EDEBUG = 0, -1, -2, -3, -4, -5, -6
PRNU_ZERO_MEAN, PRNU_WIENER_DFT, PRNU_TO_GRAY = 1, 2, 4

# every symbol declared in include/prnu.h
EXPORTS = (
    "prnu_default_params", "prnu_create", "prnu_destroy", "prnu_last_error", "prnu_workspace_size",
    "prnu_workspace_size_host", "prnu_sda_average", "prnu_denoise_residual", "prnu_fingerprint_accumulate",
    "prnu_fingerprint_accumulate_host", "prnu_fingerprint_finalize", "prnu_pce_match",
    "prnu_profile_enable", "prnu_profile_select", "prnu_profile_reset", "prnu_profile_read", "prnu_denoise_residual_static",
    "prnu_denoise_residual_batch", "prnu_pce_match_batch", "prnu_pce_match_pairs",
    "prnu_workspace_size_multi", "prnu_fingerprint_accumulate_multi", "prnu_autotune",
    "prnu_autotune_set", "prnu_sda_weighted", "prnu_sda_weighted_backward", "prnu_workspace_size_grad",
    "prnu_denoise_residual_ckpt", "prnu_denoise_residual_backward", "prnu_mle_images", "prnu_mle_images_backward",
    "prnu_workspace_size_pce_backward", "prnu_pce_backward", "prnu_workspace_size_pce_images",
    "prnu_pce_match_images", "prnu_pce_match_images_async", "prnu_pce_images_prepare",
    "prnu_pce_images_finish_async", "prnu_workspace_size_persistent", "prnu_fingerprint_accumulate_persistent",
    "prnu_persistent_status", "prnu_persistent_wait_probe", "prnu_debug_status", "prnu_autotune_level",
)


class PrnuError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libprnu status {status}: {msg}")
        self.status = status


PRNU_DTYPE_F32, PRNU_DTYPE_F16, PRNU_DTYPE_BF16 = 0, 1, 2
PRNU_FRAMES_U8, PRNU_FRAMES_F16 = 0, 1
PRNU_SDA_SEPARATE, PRNU_SDA_FUSED = -1, -2


class prnu_params(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("sigma0", ctypes.c_float), ("n_windows", ctypes.c_int),
                ("windows", ctypes.c_int * 4), ("pad_mode", ctypes.c_int), ("dtype", ctypes.c_int),
                ("frame_dtype", ctypes.c_int), ("compensated", ctypes.c_int), ("sda_blocks_per_sm", ctypes.c_int),
                ("pipeline_passes", ctypes.c_int), ("sda_fusion", ctypes.c_int)]


class prnu_camera(ctypes.Structure):
    _fields_ = [("frames", ctypes.c_void_p), ("m", ctypes.c_int), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("C", ctypes.c_int), ("frame_stride", ctypes.c_size_t), ("row_pitch", ctypes.c_size_t),
                ("d", ctypes.c_int), ("num", ctypes.c_void_p), ("den", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()
_vp, _sz, _i, _u = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint
_pp = ctypes.POINTER(prnu_params)


def _bind(path: str) -> ctypes.CDLL:
    """Load a libprnu build and declare the signature of every entry point."""
    if not os.path.exists(path):
        raise ImportError(f"{path} is not built: run __graft_entry__.build() (nvcc, sm_103a)")
    L = ctypes.CDLL(path)
    sig = {
        "prnu_default_params": [_pp],
        "prnu_create": [ctypes.POINTER(_vp), _i],
        "prnu_destroy": [_vp],
        "prnu_last_error": [_vp],
        "prnu_workspace_size": [_vp, _i, _i, _i, _pp, _i, ctypes.POINTER(_sz)],
        "prnu_workspace_size_host": [_vp, _i, _i, _i, _i, _pp, _i, ctypes.POINTER(_sz)],
        "prnu_sda_average": [_vp, _vp, _i, _i, _i, _i, _sz, _sz, _i, _vp, _vp],
        "prnu_denoise_residual": [_vp, _vp, _i, _i, _i, _pp, _vp, _vp, _sz, _vp],
        "prnu_fingerprint_accumulate": [_vp, _vp, _i, _i, _i, _i, _sz, _sz, _i, _pp, _vp, _vp, _vp, _sz, _vp],
        "prnu_fingerprint_accumulate_host": [_vp, _vp, _i, _i, _i, _i, _sz, _sz, _i, _pp, _vp, _vp, _vp,
                                             _sz, _vp],
        "prnu_fingerprint_finalize": [_vp, _vp, _vp, _i, _i, _i, _u, _pp, _vp, _vp, _sz, _vp],
        "prnu_pce_match": [_vp, _vp, _vp, _vp, _i, _i, _i, _i, ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), _vp, _sz, _vp],
        "prnu_denoise_residual_static": [_vp, _vp, _i, _i, _i, _pp, _vp, _vp],
        "prnu_denoise_residual_batch": [_vp, _vp, _i, _i, _i, _i, _pp, _vp, _vp, _sz, _vp],
        "prnu_pce_match_batch": [_vp, _vp, _vp, _vp, _i, _i, _i, _i, _i, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), _vp, _sz,
                                 _vp],
        "prnu_pce_match_pairs": [_vp, _vp, _vp, _vp, _i, _i, _i, _i, _i, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), _vp, _sz,
                                 _vp],
        "prnu_workspace_size_multi": [_vp, ctypes.POINTER(prnu_camera), _i, _pp, _i, ctypes.POINTER(_sz)],
        "prnu_fingerprint_accumulate_multi": [_vp, ctypes.POINTER(prnu_camera), _i, _pp, _vp, _sz, _vp],
        "prnu_workspace_size_persistent": [_vp, ctypes.POINTER(prnu_camera), _i, _pp, _i,
                                           ctypes.POINTER(_sz)],
        "prnu_fingerprint_accumulate_persistent": [_vp, ctypes.POINTER(prnu_camera), _i, _pp, _i,
                                                   ctypes.c_double, _vp, _sz, _vp],
        "prnu_persistent_status": [_vp, _vp, _sz, _vp, ctypes.POINTER(_i)],
        "prnu_persistent_wait_probe": [_vp, ctypes.c_double, _vp, _sz, _vp],
        "prnu_autotune": [_vp, _i, _i, _i, _pp, _i, _vp, _sz, _vp, ctypes.POINTER(_i),
                          ctypes.POINTER(ctypes.c_float)],
        "prnu_autotune_set": [_vp, _i, _i, _pp, _i],
        "prnu_autotune_level": [_vp, _i, _i, _pp, _i, _i, _i, ctypes.POINTER(_i)],
        "prnu_workspace_size_pce_images": [_vp, _i, _i, _i, _pp, _i, ctypes.POINTER(_sz)],
        "prnu_pce_match_images_async": [_vp, _vp, _vp, _i, _i, _i, _i, _pp, _i, _vp, _vp, _vp, _vp, _sz,
                                        _vp],
        "prnu_pce_images_prepare": [_vp, _vp, _i, _i, _i, _i, _pp, _vp, _sz, _vp],
        "prnu_pce_images_finish_async": [_vp, _vp, _vp, _i, _i, _i, _i, _pp, _i, _vp, _vp, _vp, _vp, _sz,
                                         _vp],
        "prnu_pce_match_images": [_vp, _vp, _vp, _i, _i, _i, _i, _pp, _i, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i), _vp, _sz, _vp],
        "prnu_sda_weighted": [_vp, _vp, _i, _i, _i, _i, _sz, _sz, _i, _vp, _vp, _vp],
        "prnu_sda_weighted_backward": [_vp, _vp, _i, _i, _i, _i, _sz, _sz, _i, _vp, _vp, _vp, _sz, _vp],
        "prnu_workspace_size_grad": [_vp, _i, _i, _i, _pp, _i, ctypes.POINTER(_sz), ctypes.POINTER(_sz)],
        "prnu_denoise_residual_ckpt": [_vp, _vp, _i, _i, _i, _i, _pp, _vp, _vp, _vp, _sz, _vp],
        "prnu_denoise_residual_backward": [_vp, _vp, _i, _i, _i, _i, _pp, _vp, _vp, _vp, _vp, _sz, _vp],
        "prnu_mle_images": [_vp, _vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, _vp, _vp],
        "prnu_mle_images_backward": [_vp, _vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp],
        "prnu_workspace_size_pce_backward": [_vp, _i, _i, _i, ctypes.POINTER(_sz)],
        "prnu_pce_backward": [_vp, _vp, _i, _vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, _vp, _vp, _sz, _vp],
        "prnu_debug_status": [_vp, ctypes.c_char_p, _sz],
        "prnu_profile_enable": [_vp, _i],
        "prnu_profile_reset": [_vp],
        "prnu_profile_select": [_vp, ctypes.c_char_p],
        "prnu_profile_read": [_vp, _i, ctypes.c_char_p, _sz, ctypes.POINTER(ctypes.c_longlong),
                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = None if name == "prnu_destroy" else (ctypes.c_char_p if name == "prnu_last_error"
                                                          else ctypes.c_int)
    return L


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(LIB_PATH)
    return _lib


def set_library(path: str | None) -> None:
    """Bind the entry points of another build of the library (the debug build
    libprnu_debug.so); None returns to the release build.  Contexts belong to
    the build that created them: close them before switching."""
    global _lib
    with _lock:
        _lib = _bind(path or LIB_PATH)


def _check(status: int, ctx=None) -> None:
    if status != PRNU_OK:
        msg = lib().prnu_last_error(ctx).decode(errors="replace")
        raise PrnuError(status, msg)


def default_params(levels=4, sigma0=3.0, windows=(3, 5, 7, 9), dtype=PRNU_DTYPE_F32, frame_dtype=PRNU_FRAMES_U8,
                   compensated=False, sda_blocks_per_sm=0, pipeline_passes=0, sda_fusion=0) -> prnu_params:
    p = prnu_params()
    _check(lib().prnu_default_params(ctypes.byref(p)))
    p.dtype = dtype
    p.frame_dtype = frame_dtype
    p.compensated = 1 if compensated else 0
    p.sda_blocks_per_sm = sda_blocks_per_sm
    p.pipeline_passes = pipeline_passes
    p.sda_fusion = sda_fusion
    p.levels = levels
    p.sigma0 = sigma0
    p.n_windows = len(windows)
    for i, w in enumerate(windows):
        p.windows[i] = w
    return p


# ------------------------------------------------------------ raw C names --
def prnu_create(device: int = 0) -> int:
    h = _vp()
    _check(lib().prnu_create(ctypes.byref(h), device))
    return h.value


def prnu_destroy(ctx: int) -> None:
    lib().prnu_destroy(ctx)


def prnu_workspace_size(ctx, H, W, C, params, images_per_pass=1) -> int:
    n = _sz()
    _check(lib().prnu_workspace_size(ctx, H, W, C, ctypes.byref(params), images_per_pass, ctypes.byref(n)), ctx)
    return n.value


def prnu_workspace_size_host(ctx, H, W, C, d, params, groups_per_pass=1) -> int:
    n = _sz()
    _check(lib().prnu_workspace_size_host(ctx, H, W, C, d, ctypes.byref(params), groups_per_pass,
                                          ctypes.byref(n)), ctx)
    return n.value


def prnu_sda_average(ctx, frames, m, H, W, C, frame_stride, row_pitch, d, sda_out, stream):
    _check(lib().prnu_sda_average(ctx, frames, m, H, W, C, frame_stride, row_pitch, d, sda_out, stream), ctx)


def prnu_denoise_residual(ctx, img, H, W, C, params, residual_out, ws, ws_bytes, stream):
    _check(lib().prnu_denoise_residual(ctx, img, H, W, C, ctypes.byref(params), residual_out, ws, ws_bytes,
                                       stream), ctx)


def prnu_denoise_residual_batch(ctx, img, n, H, W, C, params, residual_out, ws, ws_bytes, stream):
    _check(lib().prnu_denoise_residual_batch(ctx, img, n, H, W, C, ctypes.byref(params), residual_out, ws,
                                             ws_bytes, stream), ctx)


def prnu_fingerprint_accumulate(ctx, frames, m, H, W, C, frame_stride, row_pitch, d, params, num, den, ws,
                                ws_bytes, stream):
    _check(lib().prnu_fingerprint_accumulate(ctx, frames, m, H, W, C, frame_stride, row_pitch, d,
                                             ctypes.byref(params), num, den, ws, ws_bytes, stream), ctx)


def prnu_fingerprint_accumulate_host(ctx, host_frames, m, H, W, C, frame_stride, row_pitch, d, params, num, den,
                                     ws, ws_bytes, stream):
    _check(lib().prnu_fingerprint_accumulate_host(ctx, host_frames, m, H, W, C, frame_stride, row_pitch, d,
                                                  ctypes.byref(params), num, den, ws, ws_bytes, stream), ctx)


def prnu_fingerprint_finalize(ctx, num, den, H, W, C, flags, params, K_out, ws, ws_bytes, stream):
    _check(lib().prnu_fingerprint_finalize(ctx, num, den, H, W, C, flags, ctypes.byref(params), K_out, ws,
                                           ws_bytes, stream), ctx)


def prnu_pce_match(ctx, K, residual_q, img_q, H, W, C, nbhd, ws, ws_bytes, stream):
    pce, ncc = ctypes.c_double(), ctypes.c_double()
    peak = (ctypes.c_int * 2)()
    _check(lib().prnu_pce_match(ctx, K, residual_q, img_q, H, W, C, nbhd, ctypes.byref(pce), ctypes.byref(ncc),
                                peak, ws, ws_bytes, stream), ctx)
    return pce.value, ncc.value, (peak[0], peak[1])


def prnu_pce_match_batch(ctx, K, residual_q, img_q, n, H, W, C, nbhd, ws, ws_bytes, stream):
    pce = (ctypes.c_double * n)()
    ncc = (ctypes.c_double * n)()
    peak = (ctypes.c_int * (2 * n))()
    _check(lib().prnu_pce_match_batch(ctx, K, residual_q, img_q, n, H, W, C, nbhd, pce, ncc, peak, ws, ws_bytes,
                                      stream), ctx)
    return [(pce[i], ncc[i], (peak[2 * i], peak[2 * i + 1])) for i in range(n)]


def prnu_workspace_size_pce_images(ctx, H, W, C, params, n):
    b = _sz()
    _check(lib().prnu_workspace_size_pce_images(ctx, H, W, C, ctypes.byref(params), n, ctypes.byref(b)), ctx)
    return b.value


def prnu_pce_match_images(ctx, K, img_q, n, H, W, C, params, nbhd, ws, ws_bytes, stream):
    pce = (ctypes.c_double * n)()
    ncc = (ctypes.c_double * n)()
    peak = (ctypes.c_int * (2 * n))()
    _check(lib().prnu_pce_match_images(ctx, K, img_q, n, H, W, C, ctypes.byref(params), nbhd, pce, ncc, peak, ws,
                                       ws_bytes, stream), ctx)
    return [(pce[i], ncc[i], (peak[2 * i], peak[2 * i + 1])) for i in range(n)]


def prnu_pce_match_pairs(ctx, K, residual_q, img_q, n, H, W, C, nbhd, ws, ws_bytes, stream):
    pce = (ctypes.c_double * n)()
    ncc = (ctypes.c_double * n)()
    peak = (ctypes.c_int * (2 * n))()
    _check(lib().prnu_pce_match_pairs(ctx, K, residual_q, img_q, n, H, W, C, nbhd, pce, ncc, peak, ws, ws_bytes,
                                      stream), ctx)
    return [(pce[i], ncc[i], (peak[2 * i], peak[2 * i + 1])) for i in range(n)]


def prnu_denoise_residual_static(ctx, img, H, W, C, params, residual_out, stream):
    """prnu_denoise_residual with the library's fixed static scratch: no
    workspace argument and no allocation (for callers that cannot allocate)."""
    _check(lib().prnu_denoise_residual_static(ctx, img, H, W, C, ctypes.byref(params), residual_out, stream), ctx)


def prnu_workspace_size_multi(ctx, cams, params, groups_per_pass) -> int:
    arr = (prnu_camera * len(cams))(*cams)
    n = _sz()
    _check(lib().prnu_workspace_size_multi(ctx, arr, len(cams), ctypes.byref(params), groups_per_pass,
                                           ctypes.byref(n)), ctx)
    return n.value


def prnu_fingerprint_accumulate_multi(ctx, cams, params, ws, ws_bytes, stream):
    arr = (prnu_camera * len(cams))(*cams)
    _check(lib().prnu_fingerprint_accumulate_multi(ctx, arr, len(cams), ctypes.byref(params), ws, ws_bytes, stream),
           ctx)


def prnu_workspace_size_persistent(ctx, cams, params, slots=4) -> int:
    arr = (prnu_camera * len(cams))(*cams)
    n = _sz()
    _check(lib().prnu_workspace_size_persistent(ctx, arr, len(cams), ctypes.byref(params), slots, ctypes.byref(n)),
           ctx)
    return n.value


def prnu_fingerprint_accumulate_persistent(ctx, cams, params, slots, wait_budget_ms, ws, ws_bytes, stream):
    arr = (prnu_camera * len(cams))(*cams)
    _check(lib().prnu_fingerprint_accumulate_persistent(ctx, arr, len(cams), ctypes.byref(params), slots,
                                                        float(wait_budget_ms), ws, ws_bytes, stream), ctx)


def prnu_persistent_status(ctx, ws, ws_bytes, stream):
    """Synchronises the stream and returns (status, (item, group, stage)) of
    the last persistent launch in ws, without raising."""
    info = (_i * 3)()
    st = lib().prnu_persistent_status(ctx, ws, ws_bytes, stream, info)
    return st, (info[0], info[1], info[2])


def prnu_persistent_wait_probe(ctx, wait_budget_ms, ws, ws_bytes, stream):
    _check(lib().prnu_persistent_wait_probe(ctx, float(wait_budget_ms), ws, ws_bytes, stream), ctx)


STREAM_SHAPES = [(16, 4), (32, 4), (64, 4), (32, 2), (32, 8), (64, 2)]  # (strip rows, warps per block)


def prnu_autotune(ctx, H, W, C, params, images, ws, ws_bytes, stream):
    shape, ms = _i(), ctypes.c_float()
    _check(lib().prnu_autotune(ctx, H, W, C, ctypes.byref(params), images, ws, ws_bytes, stream, ctypes.byref(shape),
                               ctypes.byref(ms)), ctx)
    return shape.value, ms.value


def prnu_workspace_size_grad(ctx, H, W, C, params, n):
    ws, ck = _sz(), _sz()
    _check(lib().prnu_workspace_size_grad(ctx, H, W, C, ctypes.byref(params), n, ctypes.byref(ws), ctypes.byref(ck)),
           ctx)
    return ws.value, ck.value


def prnu_workspace_size_pce_backward(ctx, H, W, n):
    b = _sz()
    _check(lib().prnu_workspace_size_pce_backward(ctx, H, W, n, ctypes.byref(b)), ctx)
    return b.value


def call(name, ctx, *args):
    """Call a status-returning entry point of libprnu; raise PrnuError on failure."""
    _check(getattr(lib(), name)(ctx, *args), ctx)


def prnu_debug_status(ctx):
    """(status, "file:line index") of the debug build's index checks since the
    last call (synchronises the device; PRNU_EUNSUPPORTED in the release build)."""
    buf = ctypes.create_string_buffer(256)
    st = lib().prnu_debug_status(ctx, buf, 256)
    return st, buf.value.decode()


def prnu_profile_enable(ctx, on: bool) -> None:
    _check(lib().prnu_profile_enable(ctx, 1 if on else 0), ctx)


def prnu_profile_select(ctx, names=None) -> None:
    """Time only the named kernels (an iterable of profile names; None: all)."""
    _check(lib().prnu_profile_select(ctx, ",".join(names).encode() if names else None), ctx)


def prnu_profile_reset(ctx) -> None:
    _check(lib().prnu_profile_reset(ctx), ctx)


def prnu_profile_read(ctx) -> dict:
    """{kernel name: (launches, total device ms, algorithmic bytes)} since the last reset."""
    out = {}
    i = 0
    while True:
        name = ctypes.create_string_buffer(64)
        n, ms, nb = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
        st = lib().prnu_profile_read(ctx, i, name, 64, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(nb))
        if st == PRNU_EINVAL:
            break
        _check(st, ctx)
        out[name.value.decode()] = (n.value, ms.value, nb.value)
        i += 1
    return out


# ------------------------------------------------------- torch marshalling --
class Context:
    """One libprnu context on a CUDA device, with a cached workspace tensor.

    Tensors are passed by data pointer on torch's current CUDA stream.
    """

    def __init__(self, device: int = 0):
        import torch
        self.torch = torch
        self.device = device
        self.ctx = prnu_create(device)
        self._ws = None

    def close(self):
        if self.ctx:
            self.torch.cuda.synchronize(self.device)
            prnu_destroy(self.ctx)
            self.ctx = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        return self.torch.cuda.current_stream(self.device).cuda_stream

    def workspace(self, nbytes: int):
        if self._ws is None or self._ws.numel() < nbytes:
            self._ws = self.torch.empty(max(nbytes, 256), dtype=self.torch.uint8, device=f"cuda:{self.device}")
        return self._ws

    @staticmethod
    def _frames_geometry(frames):
        if frames.dim() == 3:
            frames = frames.unsqueeze(-1)
        m, H, W, C = frames.shape
        es = frames.dtype.itemsize
        assert es in (1, 2) and frames.stride(3) == 1 and frames.stride(2) == C, \
            "frames must be uint8 or float16 [m, H, W, C] with interleaved channels"
        return frames, m, H, W, C, frames.stride(0) * es, frames.stride(1) * es

    def sda_average(self, frames, d: int):
        frames, m, H, W, C, fs, rp = self._frames_geometry(frames)
        out = self.torch.empty(((m + d - 1) // d, C, H, W), dtype=self.torch.float32, device=frames.device)
        prnu_sda_average(self.ctx, frames.data_ptr(), m, H, W, C, fs, rp, d, out.data_ptr(), self._stream())
        return out

    def denoise_residual(self, img, params=None, out=None):
        params = params or default_params()
        if img.dim() == 2:
            img = img.unsqueeze(0)
        img = img.contiguous()
        C, H, W = img.shape
        out = self.torch.empty_like(img) if out is None else out
        n = prnu_workspace_size(self.ctx, H, W, C, params, 1)
        ws = self.workspace(n)
        prnu_denoise_residual(self.ctx, img.data_ptr(), H, W, C, params, out.data_ptr(), ws.data_ptr(),
                              ws.numel(), self._stream())
        return out

    def denoise_residual_batch(self, imgs, params=None, out=None):
        """imgs float32 [n, C, H, W] on the device -> residuals [n, C, H, W]."""
        params = params or default_params()
        imgs = imgs.contiguous()
        n, C, H, W = imgs.shape
        out = self.torch.empty_like(imgs) if out is None else out
        nb = prnu_workspace_size(self.ctx, H, W, C, params, n)
        ws = self.workspace(nb)
        prnu_denoise_residual_batch(self.ctx, imgs.data_ptr(), n, H, W, C, params, out.data_ptr(), ws.data_ptr(),
                                    ws.numel(), self._stream())
        return out

    def pce_match_batch(self, K, residual_q, img_q, nbhd: int = 11):
        """K [H, W]; residual_q, img_q [n, C, H, W] -> [(pce, ncc, (dy, dx))] * n."""
        n, C, H, W = residual_q.shape
        K = K.reshape(H, W).contiguous()
        nb = prnu_workspace_size(self.ctx, H, W, C, default_params(), n)
        ws = self.workspace(nb)
        return prnu_pce_match_batch(self.ctx, K.data_ptr(), residual_q.contiguous().data_ptr(),
                                    img_q.contiguous().data_ptr(), n, H, W, C, nbhd, ws.data_ptr(), ws.numel(),
                                    self._stream())

    def pce_match_images(self, K, img_q, nbhd: int = 11, params=None):
        """K [H, W]; query images [n, C, H, W] -> [(pce, ncc, (dy, dx))] * n, the
        residuals computed inside without being stored."""
        params = params or default_params()
        n, C, H, W = img_q.shape
        K = K.reshape(H, W).contiguous()
        img_q = img_q.contiguous()
        nb = prnu_workspace_size_pce_images(self.ctx, H, W, C, params, n)
        ws = self.workspace(nb)
        return prnu_pce_match_images(self.ctx, K.data_ptr(), img_q.data_ptr(), n, H, W, C, params, nbhd,
                                     ws.data_ptr(), ws.numel(), self._stream())

    def pce_match_images_async(self, K, img_q, out=None, nbhd: int = 11, params=None):
        """Like pce_match_images, with the results left on the device (no
        synchronisation; capturable in a CUDA graph after one eager call):
        returns (pce float64 [n], ncc float64 [n], peak int32 [n, 2])."""
        params = params or default_params()
        n, C, H, W = img_q.shape
        K = K.reshape(H, W)
        if out is None:
            out = (self.torch.empty(n, dtype=self.torch.float64, device=img_q.device),
                   self.torch.empty(n, dtype=self.torch.float64, device=img_q.device),
                   self.torch.empty((n, 2), dtype=self.torch.int32, device=img_q.device))
        nb = prnu_workspace_size_pce_images(self.ctx, H, W, C, params, n)
        ws = self.workspace(nb)
        _check(lib().prnu_pce_match_images_async(self.ctx, K.data_ptr(), img_q.data_ptr(), n, H, W, C,
                                                 ctypes.byref(params), nbhd, out[0].data_ptr(), out[1].data_ptr(),
                                                 out[2].data_ptr(), ws.data_ptr(), ws.numel(), self._stream()),
               self.ctx)
        return out

    def pce_images_prepare(self, img_q, params=None):
        """First half of pce_match_images_async: denoise the queries [n, C, H, W]
        down to level 2 into this context's workspace (no K needed)."""
        params = params or default_params()
        n, C, H, W = img_q.shape
        nb = prnu_workspace_size_pce_images(self.ctx, H, W, C, params, n)
        ws = self.workspace(nb)
        _check(lib().prnu_pce_images_prepare(self.ctx, img_q.data_ptr(), n, H, W, C, ctypes.byref(params),
                                             ws.data_ptr(), ws.numel(), self._stream()), self.ctx)

    def pce_images_finish_async(self, K, img_q, out=None, nbhd: int = 11, params=None):
        """Second half: grey level-1 synthesis against K and PCE, results on the
        device (pce float64 [n], ncc float64 [n], peak int32 [n, 2]); same
        img_q and the same context (workspace) as pce_images_prepare."""
        params = params or default_params()
        n, C, H, W = img_q.shape
        K = K.reshape(H, W)
        if out is None:
            out = (self.torch.empty(n, dtype=self.torch.float64, device=img_q.device),
                   self.torch.empty(n, dtype=self.torch.float64, device=img_q.device),
                   self.torch.empty((n, 2), dtype=self.torch.int32, device=img_q.device))
        nb = prnu_workspace_size_pce_images(self.ctx, H, W, C, params, n)
        ws = self.workspace(nb)
        _check(lib().prnu_pce_images_finish_async(self.ctx, K.data_ptr(), img_q.data_ptr(), n, H, W, C,
                                                  ctypes.byref(params), nbhd, out[0].data_ptr(), out[1].data_ptr(),
                                                  out[2].data_ptr(), ws.data_ptr(), ws.numel(), self._stream()),
               self.ctx)
        return out

    def pce_match_pairs(self, K, residual_q, img_q, nbhd: int = 11):
        """K [n, H, W]; residual_q, img_q [n, C, H, W]: query i against fingerprint i."""
        n, C, H, W = residual_q.shape
        nb = prnu_workspace_size(self.ctx, H, W, C, default_params(), n)
        ws = self.workspace(nb)
        return prnu_pce_match_pairs(self.ctx, K.contiguous().data_ptr(), residual_q.contiguous().data_ptr(),
                                    img_q.contiguous().data_ptr(), n, H, W, C, nbhd, ws.data_ptr(), ws.numel(),
                                    self._stream())

    def fingerprint_accumulate(self, frames, d: int, num, den, params=None, images_per_pass=None):
        """num, den: float32 [C, H, W] ([2, C, H, W] with params.compensated)."""
        params = params or default_params(frame_dtype=PRNU_FRAMES_F16 if frames.dtype.itemsize == 2 else 0)
        frames, m, H, W, C, fs, rp = self._frames_geometry(frames)
        g = (m + d - 1) // d
        n = prnu_workspace_size(self.ctx, H, W, C, params, images_per_pass or g)
        ws = self.workspace(n)
        prnu_fingerprint_accumulate(self.ctx, frames.data_ptr(), m, H, W, C, fs, rp, d, params, num.data_ptr(),
                                    den.data_ptr(), ws.data_ptr(), n, self._stream())

    def fingerprint_accumulate_host(self, host_frames, d: int, num, den, params=None, groups_per_pass=1):
        params = params or default_params(frame_dtype=PRNU_FRAMES_F16 if host_frames.dtype.itemsize == 2 else 0)
        host_frames, m, H, W, C, fs, rp = self._frames_geometry(host_frames)
        n = prnu_workspace_size_host(self.ctx, H, W, C, d, params, groups_per_pass)
        ws = self.workspace(n)
        prnu_fingerprint_accumulate_host(self.ctx, host_frames.data_ptr(), m, H, W, C, fs, rp, d, params,
                                         num.data_ptr(), den.data_ptr(), ws.data_ptr(), n, self._stream())

    def autotune(self, H, W, C, params=None, images=4):
        """Pick the level-1 analysis launch shape for this geometry; returns
        ((strip rows, warps), ms per launch)."""
        params = params or default_params()
        n = prnu_workspace_size(self.ctx, H, W, C, params, images)
        ws = self.workspace(n)
        shape, ms = prnu_autotune(self.ctx, H, W, C, params, images, ws.data_ptr(), n, self._stream())
        return STREAM_SHAPES[shape], ms

    def autotune_set(self, H, W, shape, params=None):
        """Pin the level-1 analysis shape (index into STREAM_SHAPES; -1 = default)."""
        _check(lib().prnu_autotune_set(self.ctx, H, W, ctypes.byref(params or default_params()), shape), self.ctx)

    def autotune_level(self, H, W, kind, level, choice=-2, params=None):
        """Pin (choice >= 0), reset (-1) or read (-2) the tuner's choice for a
        launch kind (0 analysis, 1 shrink, 2 synthesis, 3 the level-1 MLE step)
        at a level; returns the choice in force."""
        cur = _i()
        _check(lib().prnu_autotune_level(self.ctx, H, W, ctypes.byref(params or default_params()), kind, level,
                                         choice, ctypes.byref(cur)), self.ctx)
        return cur.value

    def cameras(self, items):
        """[(frames [m, H, W, C] tensor, d, num, den)] -> prnu_camera structs."""
        out = []
        for frames, d, num, den in items:
            frames, m, H, W, C, fs, rp = self._frames_geometry(frames)
            out.append(prnu_camera(frames.data_ptr(), m, H, W, C, fs, rp, d, num.data_ptr(), den.data_ptr()))
        return out

    def fingerprint_accumulate_multi(self, items, params=None, groups_per_pass=64, ws_bytes=None):
        """items: [(frames, d, num, den)] of several cameras (any geometries)."""
        params = params or default_params(frame_dtype=PRNU_FRAMES_F16 if items[0][0].dtype.itemsize == 2 else 0)
        cams = self.cameras(items)
        n = ws_bytes or prnu_workspace_size_multi(self.ctx, cams, params, groups_per_pass)
        ws = self.workspace(n)
        prnu_fingerprint_accumulate_multi(self.ctx, cams, params, ws.data_ptr(), n, self._stream())

    def fingerprint_accumulate_persistent(self, items, params=None, slots=4, wait_budget_ms=2000.0, check=True):
        """items: [(frames, d, num, den)] of several cameras (any geometries),
        in one persistent launch; with check=True the queue status is read
        back (synchronising) and a timed-out wait raises PrnuError."""
        params = params or default_params()
        cams = self.cameras(items)
        n = prnu_workspace_size_persistent(self.ctx, cams, params, slots)
        ws = self.workspace(n)
        prnu_fingerprint_accumulate_persistent(self.ctx, cams, params, slots, wait_budget_ms, ws.data_ptr(), n,
                                               self._stream())
        if check:
            st, info = prnu_persistent_status(self.ctx, ws.data_ptr(), n, self._stream())
            _check(st, self.ctx)

    def fingerprint_finalize(self, num, den, flags: int = 0, params=None):
        params = params or default_params()
        C, H, W = num.shape[-3:]
        Cout = 1 if flags & PRNU_TO_GRAY else C
        K = self.torch.empty((Cout, H, W), dtype=self.torch.float32, device=num.device)
        n = prnu_workspace_size(self.ctx, H, W, C, params, 1)
        ws = self.workspace(n)
        prnu_fingerprint_finalize(self.ctx, num.data_ptr(), den.data_ptr(), H, W, C, flags, params, K.data_ptr(),
                                  ws.data_ptr(), ws.numel(), self._stream())
        return K

    def pce_match(self, K, residual_q, img_q, nbhd: int = 11):
        if residual_q.dim() == 2:
            residual_q, img_q = residual_q.unsqueeze(0), img_q.unsqueeze(0)
        C, H, W = residual_q.shape
        K = K.reshape(H, W).contiguous()
        n = prnu_workspace_size(self.ctx, H, W, C, default_params(), 1)
        ws = self.workspace(n)
        return prnu_pce_match(self.ctx, K.data_ptr(), residual_q.contiguous().data_ptr(),
                              img_q.contiguous().data_ptr(), H, W, C, nbhd, ws.data_ptr(), ws.numel(),
                              self._stream())
