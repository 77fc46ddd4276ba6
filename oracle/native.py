"""Build and load the plain-C FP64 core of the oracle (oracle/prnu_oracle.c).

TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the CPU
legs of bench.py; never by the CUDA product path.

The shared object is compiled with the host gcc on first use (and by
__graft_entry__.build()).  OpenMP is used when the compiler supports it; every
parallel loop in the C file writes disjoint outputs, so results do not depend
on the thread count.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "prnu_oracle.c")
_LIB = os.path.join(_HERE, "_prnu_oracle.so")
_lock = threading.Lock()
_lib = None
_openmp = False


def build(force: bool = False) -> str:
    """Compile prnu_oracle.c into _prnu_oracle.so (with OpenMP if available)."""
    global _openmp
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        _openmp = _probe_openmp_flag()
        return _LIB
    base = ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", _LIB + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
        _openmp = True
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
        _openmp = False
    os.replace(_LIB + ".tmp", _LIB)
    with open(_LIB + ".omp", "w") as f:
        f.write("1" if _openmp else "0")
    return _LIB


def _probe_openmp_flag() -> bool:
    try:
        with open(_LIB + ".omp") as f:
            return f.read().strip() == "1"
    except OSError:
        return False


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            L.orc_sda_average.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_long, ctypes.c_long, ctypes.c_int, dp]
            L.orc_pad_mirror.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
            L.orc_dwt2_level.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp, dp, dp, dp]
            L.orc_idwt2_level.argtypes = [dp, dp, dp, dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp]
            L.orc_shrink_subband.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ip,
                                             ctypes.c_int, dp, dp, dp]
            L.orc_denoise_plane.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int,
                                            ctypes.c_double, ip, ctypes.c_int, dp, dp]
            L.orc_residual_plane.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int,
                                             ctypes.c_double, ip, ctypes.c_int, dp]
            L.orc_mle_accumulate.argtypes = [dp, dp, ctypes.c_long, dp, dp]
            L.orc_mle_finalize.argtypes = [dp, dp, ctypes.c_long, dp]
            for name in ("orc_sda_average", "orc_pad_mirror", "orc_dwt2_level", "orc_idwt2_level",
                         "orc_shrink_subband", "orc_denoise_plane", "orc_residual_plane"):
                getattr(L, name).restype = ctypes.c_int
            L.orc_mle_accumulate.restype = None
            L.orc_mle_finalize.restype = None
            _lib = L
    return _lib


_threads_set = None


def threads() -> int:
    """Threads the C core runs with (1 when built without OpenMP)."""
    lib()
    if not _openmp:
        return 1
    if _threads_set:
        return _threads_set
    n = os.environ.get("OMP_NUM_THREADS")
    if n:
        return int(n)
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def set_threads(n: int | None) -> int:
    """Run the C core's parallel loops on n threads (None: back to the
    default, all cores of the affinity mask); returns the count in effect.
    Results do not depend on it (every parallel loop writes disjoint
    outputs)."""
    global _threads_set
    L = lib()
    if not _openmp:
        return 1
    fn = getattr(L, "omp_set_num_threads", None)  # from the OpenMP runtime the library links
    if fn is None:  # pragma: no cover
        return threads()
    _threads_set = None
    want = int(n) if n else threads()
    fn(ctypes.c_int(want))
    _threads_set = int(n) if n else None
    return threads()


def dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def iptr(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")
