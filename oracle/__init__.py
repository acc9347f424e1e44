"""FP64 CPU oracle for the hop-size CWT (CWTH).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(``paper_2408_14302_gb300``) never does, and the two share no code.

The arithmetic lives in ``cwth_oracle.c`` (plain C, float64, OpenMP over
frames): the discretised Eq. 1 of the paper (Sec. II.A) evaluated only at the
positions b = k*H (Sec. II.B), with the complex Morlet wavelet
psi(t) = (pi*B)^{-1/2} exp(-t^2/B) exp(i 2 pi C t).  This module is a ctypes
shim plus the compiler call that builds it.

Every function is pinned by ``tests/test_oracle_pins.py`` against things the
definition fixes independently of this code: the closed-form response to a
complex exponential (Poisson-summed Morlet spectrum), bitwise hop decimation
and shift invariance, linearity, time reversal, a pure-Python brute force of
Eq. 1 on tiny inputs and a numpy-FFT evaluation of the same convolution.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cwth_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

_lock = threading.Lock()
_lib = None

# Truncation used by default: taps below 1e-16 of the wavelet peak are dropped.
DEFAULT_EPS = 1e-16


def build(force: bool = False) -> str:
    """Compile ``cwth_oracle.c`` with gcc into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
           "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_cwth.argtypes = [
                dp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, dp,
                ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                ctypes.c_int32, dp, dp, dp]
            lib.oracle_cwth.restype = ctypes.c_int
            lib.oracle_half_support.argtypes = [ctypes.c_double, ctypes.c_double,
                                                ctypes.c_double]
            lib.oracle_half_support.restype = ctypes.c_int64
            lib.oracle_num_frames.argtypes = [ctypes.c_int64, ctypes.c_int32]
            lib.oracle_num_frames.restype = ctypes.c_int64
            lib.oracle_max_threads.argtypes = []
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_frames(n: int, hop: int) -> int:
    """F = ceil(n / hop): frames at b = 0, H, 2H, ... inside [0, n)."""
    return int(_load().oracle_num_frames(int(n), int(hop)))


def half_support(a: float, bandwidth: float, eps: float = DEFAULT_EPS) -> int:
    """h = ceil(a * sqrt(B ln(1/eps))), the oracle's truncation radius."""
    return int(_load().oracle_half_support(float(a), float(bandwidth), float(eps)))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def cwth(x, scales, hop: int, bandwidth: float = 1.5, center: float = 1.0,
         eps: float = DEFAULT_EPS, truncate: bool = True, threads: int = 0):
    """Complex CWTH coefficients W[s, k] of one real signal, float64.

    ``x``: 1-D real signal; ``scales``: scales in samples; returns a complex128
    array of shape [S, ceil(len(x)/hop)].
    """
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
    sc = np.ascontiguousarray(np.asarray(scales, dtype=np.float64).ravel())
    n, S = x.shape[0], sc.shape[0]
    if n <= 0 or S <= 0 or int(hop) <= 0:
        raise ValueError("oracle.cwth needs a non-empty signal, scales and hop >= 1")
    F = num_frames(n, hop)
    re = np.empty((S, F), np.float64)
    im = np.empty((S, F), np.float64)
    rc = _load().oracle_cwth(_dptr(x), n, float(bandwidth), float(center), _dptr(sc),
                             S, int(hop), float(eps), 1 if truncate else 0,
                             int(threads), _dptr(re), _dptr(im),
                             ctypes.POINTER(ctypes.c_double)())
    if rc != 0:
        raise ValueError(f"oracle_cwth rejected its arguments (rc={rc})")
    return re + 1j * im


def cwth_resampled(x, scales, hop: int, **kw):
    """Resample-first reading of the hop (paper Sec. III.B and Fig. 2, the
    alternative to the output decimation of Sec. II.B): the signal is
    re-sampled at the hop spacing, y[m] = x[m hop] for m < ceil(n / hop),
    and Eq. 1 is evaluated at every sample of y with scales a / hop.
    Complex [S, ceil(n / hop)], float64."""
    h = int(hop)
    y = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel()[::h])
    return cwth(y, np.asarray(scales, dtype=np.float64) / h, 1, **kw)


def cwth_magnitude(x, scales, hop: int, **kw):
    """|W[s, k]| of one real signal, float64 (the scalogram)."""
    return np.abs(cwth(x, scales, hop, **kw))
