"""Build and load the oracle's plain-C loops (``ref_native.c``) through ctypes.

Test infrastructure only.  The flags switch off multiply-add contraction
(``-ffp-contract=off``), because the brute-force neighbour decision relies on
one fixed rounding per operation.  Nothing architecture specific is used, so
the same source builds on x86-64 and on aarch64.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ref_native.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to its source if it is missing or stale."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I8 = ctypes.POINTER(ctypes.c_int8)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.or_pairs_count.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_double, _I32, _I64]
            L.or_pairs_fill.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_double, _I32, _I64,
                                        _I32, _I8]
            L.or_realspace_brute.argtypes = [ctypes.c_int64, _D, _D, _D, _D, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int64, _I64, _D, _D]
            L.or_realspace_matrix.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_double,
                                              ctypes.c_double, _D]
            L.or_realspace_cells.argtypes = [ctypes.c_int64, _D, _D, _D, _D, ctypes.c_double,
                                             ctypes.c_double, _D, _D]
            L.or_ewald_kspace.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_double,
                                          ctypes.c_double, _D, _D, _D]
            L.or_num_threads.restype = ctypes.c_int
            _lib = L
        return _lib


def dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def i64ptr(a: np.ndarray):
    assert a.dtype == np.int64 and a.flags.c_contiguous
    return a.ctypes.data_as(_I64)


def i32ptr(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(_I32)


def i8ptr(a: np.ndarray):
    assert a.dtype == np.int8 and a.flags.c_contiguous
    return a.ctypes.data_as(_I8)


def num_threads() -> int:
    return int(lib().or_num_threads())
