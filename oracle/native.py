"""Builds and loads the oracle's small C helper (exact int64 8-bit Gram).

Test infrastructure only (see oracle/__init__.py). Compiled with the host gcc,
no architecture-specific flags, so the same source builds on x86_64 and Arm.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gram_u8.c")
_LIB = os.path.join(_HERE, "_oracle_gram_u8.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile oracle/gram_u8.c into oracle/_oracle_gram_u8.so (idempotent)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC]
    try:
        subprocess.check_call(cmd)
    except (OSError, subprocess.CalledProcessError):
        # OpenMP is a convenience for the timed baseline, not part of the result.
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC]
        subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.oracle_dot_u8.restype = ctypes.c_int64
            L.oracle_dot_u8.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
            L.oracle_gram_u8.restype = None
            L.oracle_gram_u8.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                         ctypes.c_void_p]
            L.oracle_num_threads.restype = ctypes.c_int
            L.oracle_num_threads.argtypes = []
            _lib = L
    return _lib


def num_threads():
    return int(lib().oracle_num_threads())


def gram_u8_cols(cols):
    """Exact int64 Gram of a list of equal-length uint8 vectors."""
    cols = [np.ascontiguousarray(c, dtype=np.uint8).reshape(-1) for c in cols]
    c = len(cols)
    G = np.zeros((c, c), dtype=np.int64)
    if c == 0:
        return G
    n = cols[0].size
    for v in cols:
        if v.size != n:
            raise ValueError("snapshots differ in length")
    ptrs = (ctypes.c_void_p * c)(*[v.ctypes.data for v in cols])
    lib().oracle_gram_u8(ptrs, n, c, G.ctypes.data)
    return G


def dot_u8(a, b):
    a = np.ascontiguousarray(a, dtype=np.uint8).reshape(-1)
    b = np.ascontiguousarray(b, dtype=np.uint8).reshape(-1)
    if a.size != b.size:
        raise ValueError("length mismatch")
    return int(lib().oracle_dot_u8(a.ctypes.data, b.ctypes.data, a.size))
