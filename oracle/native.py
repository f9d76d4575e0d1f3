"""Builds and loads the oracle's small C helpers: the exact int64 8-bit Gram
(gram_u8.c) and the streaming Gram update on the host cores (stream_cpu.c,
the timed streaming CPU baseline).

Test infrastructure only (see oracle/__init__.py). Compiled with the host gcc,
no architecture-specific flags, so the same sources build on x86_64 and Arm.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "gram_u8.c"), os.path.join(_HERE, "stream_cpu.c")]
_LIB = os.path.join(_HERE, "_oracle_gram_u8.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle's C sources into oracle/_oracle_gram_u8.so (idempotent)."""
    if (not force and os.path.exists(_LIB)
            and all(os.path.getmtime(_LIB) >= os.path.getmtime(src) for src in _SRCS)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O3", "-fPIC", "-shared", "-fopenmp", "-o", tmp] + _SRCS
    try:
        subprocess.check_call(cmd)
    except (OSError, subprocess.CalledProcessError):
        # OpenMP is a convenience for the timed baselines, not part of the result.
        cmd = ["gcc", "-O3", "-fPIC", "-shared", "-o", tmp] + _SRCS
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
            L.scpu_threads.restype = ctypes.c_int
            L.scpu_threads.argtypes = []
            for name in ("scpu_push_u8", "scpu_push_f32"):
                f = getattr(L, name)
                f.restype = ctypes.c_int
                f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                              ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
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


class StreamingCPU:
    """The streaming Gram update on the host cores (stream_cpu.c): a ring of m
    slots of n elements and the physical Gram G (m x m). push(x) writes x into
    the next slot (the oldest once the window is full) and sets G's row and
    column of that slot to the new inner products."""

    def __init__(self, n, m, kind="u8"):
        if kind not in ("u8", "f32"):
            raise ValueError(kind)
        self.n, self.m, self.kind = int(n), int(m), kind
        dt = np.uint8 if kind == "u8" else np.float32
        self.ring = np.zeros((self.m, self.n), dtype=dt)
        self.G = np.zeros((self.m, self.m), dtype=np.int64 if kind == "u8" else np.float64)
        self.count = 0

    def fill(self, frames):
        """Load a full window without computing G (for timing runs, where G's
        content does not matter): slot s takes frames[s % len(frames)]."""
        for s in range(self.m):
            self.ring[s] = frames[s % len(frames)]
        self.count = self.m

    def push(self, x):
        x = np.ascontiguousarray(x, dtype=self.ring.dtype).reshape(-1)
        if x.size != self.n:
            raise ValueError("snapshot length %d, expected %d" % (x.size, self.n))
        s_new = self.count % self.m
        used = min(self.count + 1, self.m)
        f = lib().scpu_push_u8 if self.kind == "u8" else lib().scpu_push_f32
        rc = f(self.ring.ctypes.data, self.n, self.n, self.m, used, s_new, x.ctypes.data,
               self.G.ctypes.data)
        if rc != 0:
            raise ValueError("scpu push rejected its arguments")
        self.count += 1
        return s_new


def scpu_threads():
    return int(lib().scpu_threads())
