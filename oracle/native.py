"""Build and load the oracle's plain-C loops (test infrastructure only).

Compiled with gcc, -O2, OpenMP, and -ffp-contract=off so that no
multiply-add is fused: the oracle's FP64 arithmetic is exactly the IEEE
sequence written in the source, on x86-64 and on aarch64 alike.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "oracle_sums.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle_sums.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile oracle_sums.c into oracle/_build/liboracle_sums.so (idempotent)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.oracle_punctured_sum.argtypes = [ctypes.c_int64, _D, _D, _D, _D, _D, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, _I, _I, _I,
                                               ctypes.c_int64, _D, _D]
            L.oracle_punctured_sum.restype = None
            L.oracle_reaction_potential.argtypes = [ctypes.c_int64, _D, _D, _D, _D, _D, ctypes.c_double,
                                                    ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                                    _D, _D]
            L.oracle_reaction_potential.restype = None
            L.oracle_cutoff_g.argtypes = [ctypes.c_double, ctypes.c_double]
            L.oracle_cutoff_g.restype = ctypes.c_double
            L.oracle_punctured_lattice_many.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_double,
                                                        ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                                        _D, _D]
            L.oracle_punctured_lattice_many.restype = None
            L.oracle_tree_near.argtypes = [ctypes.c_int64, _D, _D, _D, _D, _D, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, _I, _I, _I, ctypes.c_int64, _I, _I, _D, _D]
            L.oracle_tree_near.restype = None
            L.oracle_tree_far.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_double, _I, ctypes.c_int64, _I, _I,
                                          ctypes.c_int64, _D, _D, _D, _D]
            L.oracle_tree_far.restype = None
            L.oracle_set_threads.argtypes = [ctypes.c_int]
            L.oracle_set_threads.restype = None
            L.oracle_max_threads.argtypes = []
            L.oracle_max_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def iptr(a: np.ndarray):
    assert a.dtype == np.int64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_I)


def set_threads(n: int | None):
    """Set the OpenMP thread count for subsequent oracle calls (None: leave default)."""
    if n is not None:
        lib().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(lib().oracle_max_threads())
