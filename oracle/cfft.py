"""ctypes front end of the oracle's plain C transforms (``fft3.c``).

TEST INFRASTRUCTURE ONLY: part of the CPU oracle.  Only ``tests/``, the smoke
check and the benchmark's CPU-baseline leg may import it.

The shared object is compiled with gcc on first use (or by ``build()``), into
this directory, from ``fft3.c`` alone.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fft3.c")
_LIB = os.path.join(_HERE, "liboracle_fft.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``fft3.c`` into ``liboracle_fft.so`` (OpenMP if gcc supports it)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.c_void_p
            ci = ctypes.c_int
            lib.oracle_dft1d.argtypes = [dp, dp, ci, ci]
            lib.oracle_fft1d.argtypes = [dp, dp, ci, ci]
            lib.oracle_fft3d.argtypes = [dp, ci, ci, ci, ci, ci]
            lib.oracle_dft3d_direct.argtypes = [dp, dp, ci, ci, ci, ci]
            lib.oracle_num_threads.restype = ci
            _lib = lib
    return _lib


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def dft1d(x, sign: int) -> np.ndarray:
    """Direct O(n^2) sum  y[m] = sum_t x[t] exp(sign 2 pi i t m / n)."""
    x = _c128(x)
    y = np.empty_like(x)
    _load().oracle_dft1d(x.ctypes.data, y.ctypes.data, x.size, int(sign))
    return y


def fft1d(x, sign: int) -> np.ndarray:
    """Recursive Cooley-Tukey transform with the same definition as dft1d."""
    x = _c128(x)
    y = np.empty_like(x)
    _load().oracle_fft1d(x.ctypes.data, y.ctypes.data, x.size, int(sign))
    return y


def fft3d(a, sign: int) -> np.ndarray:
    """Unnormalised 3-D transform over the last three axes of ``a``.

    Leading axes are independent boxes.  Returns a new array.
    """
    a = np.array(a, dtype=np.complex128, order="C", copy=True)
    S0, S1, S2 = a.shape[-3:]
    count = int(np.prod(a.shape[:-3], dtype=np.int64)) if a.ndim > 3 else 1
    _load().oracle_fft3d(a.ctypes.data, S0, S1, S2, count, int(sign))
    return a


def dft3d_direct(a, sign: int) -> np.ndarray:
    """O(N^2) 3-D sum over one box (tiny boxes only)."""
    a = _c128(a)
    assert a.ndim == 3
    y = np.empty_like(a)
    _load().oracle_dft3d_direct(a.ctypes.data, y.ctypes.data, *a.shape, int(sign))
    return y


def num_threads() -> int:
    """OpenMP threads the per-axis loops use (1 without OpenMP)."""
    return int(_load().oracle_num_threads())
