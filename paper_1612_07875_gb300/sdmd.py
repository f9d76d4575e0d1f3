"""Thin ctypes binding of libsdmd (include/sdmd.h): same names, argument
marshalling only. Every step of the computation runs in the library's CUDA
kernels; there is no Python or CPU fallback. If libsdmd.so is missing or
cannot be loaded, the first call raises.

Pointer arguments accept a torch tensor, a numpy array, or a raw address
(int). Streams accept a torch.cuda.Stream, a raw cudaStream_t (int) or
None / 0 for the legacy default stream.
"""
import ctypes
import os
import threading

SDMD_F32 = 0
SDMD_U8 = 1
SDMD_C64 = 2
SDMD_C64_SPARSE = 3

SDMD_OK = 0
SDMD_ERR_ARG = -1
SDMD_ERR_OOM = -2
SDMD_ERR_NOT_READY = -3
SDMD_ERR_CUDA = -4
SDMD_ERR_TIMEOUT = -5
SDMD_ERR_RANK = -6
SDMD_ERR_UNSUPPORTED = -7
SDMD_MAX_M = 256
SDMD_MAX_DEPTH = 16

SDMD_OPT_PHI_TENSOR = 1
SDMD_OPT_REBUILD_TENSOR = 2
SDMD_OPT_F32_BF16X3 = 3
SDMD_OPT_F32_FP64 = 4
SDMD_OPT_HOST_EARLY_READ = 5

SDMD_RECON_MODES = 0
SDMD_RECON_BACKGROUND = 1
SDMD_RECON_FOREGROUND = 2
SDMD_RECON_BACKGROUND_SLOW = 3
SDMD_RECON_FOREGROUND_SLOW = 4

SDMD_K_INGEST = 0
SDMD_K_GRAM_ROW = 1
SDMD_K_MODES = 2
SDMD_K_PHI = 3
SDMD_K_FRAME = 4
SDMD_K_FUSED = 5
SDMD_K_COUNT = 6

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsdmd.so")

_lock = threading.Lock()
_lib = None

_VP = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32

# name -> argtypes (every entry point returns int except sdmd_last_error)
_SIGNATURES = {
    "sdmd_create": [_I64, _I32, _I32, ctypes.POINTER(_VP)],
    "sdmd_destroy": [_VP],
    "sdmd_create_ex": [_I64, _I32, _I32, _I32, ctypes.POINTER(_VP)],
    "sdmd_step": [_VP, _VP, _I32, _VP, _VP, _VP, _VP],
    "sdmd_sync": [_VP, _VP],
    "sdmd_set_option": [_VP, _I32, _I64],
    "sdmd_trace_times": [_VP, _I32, ctypes.POINTER(ctypes.c_double), _I32, ctypes.POINTER(_I32)],
    "sdmd_create_sparse": [_I64, _I32, _I32, ctypes.POINTER(_VP)],
    "sdmd_push_sparse": [_VP, _I32, _VP, _VP, _VP],
    "sdmd_push": [_VP, _VP, _VP],
    "sdmd_count": [_VP, ctypes.POINTER(_I64)],
    "sdmd_rebuild": [_VP, _VP],
    "sdmd_gram": [_VP, _VP, _VP],
    "sdmd_newest_row": [_VP, _VP, _VP],
    "sdmd_modes_many": [ctypes.POINTER(_VP), _I32, ctypes.POINTER(_I32), ctypes.POINTER(_VP), _VP, _VP],
    "sdmd_set_newest_row": [_VP, _VP, _VP],
    "sdmd_modes": [_VP, _I32, _VP, _VP, _VP, _VP],
    "sdmd_svd": [_VP, _I32, _VP, _VP, _VP],
    "sdmd_status": [_VP, _VP],
    "sdmd_trace": [_VP, _I32],
    "sdmd_trace_read": [_VP, _I32, ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_double)],
    "sdmd_gram_row_static": [_I32, _VP, _I64, _I32, _VP, _I64, _VP, _VP],
    "sdmd_modes_phase_cycles": [_VP, ctypes.POINTER(_I64), _I32, _VP],
    "sdmd_amplitudes": [_VP, _VP, ctypes.POINTER(_I32), _VP],
    "sdmd_push_batch": [_VP, _I32, _VP, _I64, _VP],
    "sdmd_push_many": [ctypes.POINTER(_VP), ctypes.POINTER(_VP), _I32, _VP],
    "sdmd_server_create": [_I64, ctypes.POINTER(_VP)],
    "sdmd_server_destroy": [_VP],
    "sdmd_server_stream": [_VP, ctypes.POINTER(_VP)],
    "sdmd_server_open": [_VP, _I64, _I32, _I32, ctypes.POINTER(_I32)],
    "sdmd_server_state": [_VP, _I32],
    "sdmd_server_handle": [_VP, _I32, ctypes.POINTER(_VP)],
    "sdmd_server_submit": [_VP, _I32, _VP, ctypes.c_double],
    "sdmd_server_tick": [_VP, ctypes.POINTER(_I32)],
    "sdmd_server_close": [_VP, _I32],
    "sdmd_server_stats": [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64)],
    "sdmd_server_used_bytes": [_VP],
    "sdmd_server_reset_stats": [_VP],
    "sdmd_server_set_graphs": [_VP, _I32],
    "sdmd_server_graph_stats": [_VP, ctypes.POINTER(_I64), ctypes.POINTER(_I64)],
    "sdmd_server_autotune": [_VP],
    "sdmd_server_clock_ms": [],
    "sdmd_reconstruct": [_VP, _I64, _I32, _VP, _VP],
    "sdmd_reconstruct_ex": [_VP, _I64, _I32, ctypes.c_double, _VP, _VP],
    "sdmd_pod_modes": [_VP, _I32, _VP, _VP],
    "sdmd_fourier_modes": [_VP, _I32, _VP, _VP, _I64, ctypes.POINTER(_I64), _VP],
    "sdmd_autotune": [_VP, ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_double), _VP],
}


class SdmdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (status %d)" % (msg, code))
        self.code = code


def lib():
    """Load libsdmd.so (raises if it is not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libsdmd.so is not built (%s); run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            for name, argt in _SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = argt
                fn.restype = ctypes.c_int
            L.sdmd_last_error.argtypes = []
            L.sdmd_last_error.restype = ctypes.c_char_p
            L.sdmd_server_used_bytes.restype = ctypes.c_int64
            L.sdmd_server_clock_ms.restype = ctypes.c_double
            _lib = L
    return _lib


def ptr(x):
    """Address of a torch tensor / numpy array / int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError("cannot take the address of %r" % type(x))


def stream_handle(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    raise TypeError("not a stream: %r" % type(s))


def _check(rc, fn):
    if rc != SDMD_OK:
        raise SdmdError(rc, "%s: %s" % (fn, sdmd_last_error()))
    return rc


def sdmd_last_error():
    return lib().sdmd_last_error().decode(errors="replace")


def sdmd_create(n, m, dtype):
    h = _VP()
    _check(lib().sdmd_create(int(n), int(m), int(dtype), ctypes.byref(h)), "sdmd_create")
    return h.value


def sdmd_create_ex(n, m, dtype, depth):
    h = _VP()
    _check(lib().sdmd_create_ex(int(n), int(m), int(dtype), int(depth), ctypes.byref(h)), "sdmd_create_ex")
    return h.value


def sdmd_step(h, x, r, phi, lam, r_out=None, stream=None):
    _check(lib().sdmd_step(h, ptr(x), int(r), ptr(phi), ptr(lam), ptr(r_out), stream_handle(stream)), "sdmd_step")


def sdmd_sync(h, stream=None):
    _check(lib().sdmd_sync(h, stream_handle(stream)), "sdmd_sync")


def sdmd_create_sparse(n, m, nnz_max):
    h = _VP()
    _check(lib().sdmd_create_sparse(int(n), int(m), int(nnz_max), ctypes.byref(h)), "sdmd_create_sparse")
    return h.value


def sdmd_push_sparse(h, nnz, idx, vals, stream=None):
    _check(lib().sdmd_push_sparse(h, int(nnz), ptr(idx), ptr(vals), stream_handle(stream)), "sdmd_push_sparse")


def sdmd_destroy(h):
    _check(lib().sdmd_destroy(h), "sdmd_destroy")


def sdmd_push(h, x, stream=None):
    _check(lib().sdmd_push(h, ptr(x), stream_handle(stream)), "sdmd_push")


def sdmd_rebuild(h, stream=None):
    _check(lib().sdmd_rebuild(h, stream_handle(stream)), "sdmd_rebuild")


def sdmd_count(h):
    c = _I64()
    _check(lib().sdmd_count(h, ctypes.byref(c)), "sdmd_count")
    return c.value


def sdmd_gram(h, G, stream=None):
    _check(lib().sdmd_gram(h, ptr(G), stream_handle(stream)), "sdmd_gram")


def sdmd_modes_many(hs, r, lambdas=None, r_out=None, stream=None):
    """Eigensolvers of several handles in one launch (see sdmd.h); r is one
    int or a list, lambdas a list of per-handle buffers (or None)."""
    count = len(hs)
    rr = [int(r)] * count if isinstance(r, int) else [int(x) for x in r]
    harr = (_VP * count)(*hs)
    rarr = (_I32 * count)(*rr)
    larr = (_VP * count)(*[ptr(x) for x in lambdas]) if lambdas is not None else None
    _check(lib().sdmd_modes_many(harr, count, rarr, larr, ptr(r_out), stream_handle(stream)), "sdmd_modes_many")


def sdmd_newest_row(h, row, stream=None):
    """The newest snapshot's row of G, time order (c values; see sdmd.h)."""
    _check(lib().sdmd_newest_row(h, ptr(row), stream_handle(stream)), "sdmd_newest_row")


def sdmd_set_newest_row(h, row, stream=None):
    """Overwrite the newest snapshot's row and column of G (time order)."""
    _check(lib().sdmd_set_newest_row(h, ptr(row), stream_handle(stream)), "sdmd_set_newest_row")


def sdmd_modes(h, r, phi, lam, r_out=None, stream=None):
    _check(lib().sdmd_modes(h, int(r), ptr(phi), ptr(lam), ptr(r_out), stream_handle(stream)),
           "sdmd_modes")


def sdmd_svd(h, r, sigma, V, stream=None):
    _check(lib().sdmd_svd(h, int(r), ptr(sigma), ptr(V), stream_handle(stream)), "sdmd_svd")


def sdmd_push_batch(h, k, X, ld, stream=None):
    """Append k snapshots (snapshot j at X + j * ld elements)."""
    _check(lib().sdmd_push_batch(h, int(k), ptr(X), int(ld), stream_handle(stream)), "sdmd_push_batch")


SDMD_MAX_BATCH = 64


def sdmd_push_many(hs, xs, stream=None):
    """One snapshot per handle, all Gram rows in one launch."""
    k = len(hs)
    harr = (_VP * k)(*hs)
    xarr = (_VP * k)(*[ptr(x) for x in xs])
    _check(lib().sdmd_push_many(harr, xarr, k, stream_handle(stream)), "sdmd_push_many")


SDMD_STREAM_WAITING = 0
SDMD_STREAM_ACTIVE = 1
SDMD_STREAM_CLOSED = 2


def sdmd_server_create(hbm_budget):
    s = _VP()
    _check(lib().sdmd_server_create(int(hbm_budget), ctypes.byref(s)), "sdmd_server_create")
    return s.value


def sdmd_server_destroy(s):
    _check(lib().sdmd_server_destroy(s), "sdmd_server_destroy")


def sdmd_server_stream(s):
    st = _VP()
    _check(lib().sdmd_server_stream(s, ctypes.byref(st)), "sdmd_server_stream")
    return st.value


def sdmd_server_open(s, n, m, dtype):
    sid = _I32()
    _check(lib().sdmd_server_open(s, int(n), int(m), int(dtype), ctypes.byref(sid)), "sdmd_server_open")
    return sid.value


def sdmd_server_state(s, sid):
    rc = lib().sdmd_server_state(s, int(sid))
    if rc < 0:
        _check(rc, "sdmd_server_state")
    return rc


def sdmd_server_handle(s, sid):
    h = _VP()
    _check(lib().sdmd_server_handle(s, int(sid), ctypes.byref(h)), "sdmd_server_handle")
    return h.value


def sdmd_server_submit(s, sid, x, arrival_ms=-1.0):
    _check(lib().sdmd_server_submit(s, int(sid), ptr(x), float(arrival_ms)), "sdmd_server_submit")


def sdmd_server_tick(s):
    n = _I32()
    _check(lib().sdmd_server_tick(s, ctypes.byref(n)), "sdmd_server_tick")
    return n.value


def sdmd_server_close(s, sid):
    _check(lib().sdmd_server_close(s, int(sid)), "sdmd_server_close")


def sdmd_server_stats(s):
    """(p50_ms, p99_ms, frames)"""
    p50, p99, fr = ctypes.c_double(), ctypes.c_double(), _I64()
    _check(lib().sdmd_server_stats(s, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(fr)), "sdmd_server_stats")
    return p50.value, p99.value, fr.value


def sdmd_server_used_bytes(s):
    return lib().sdmd_server_used_bytes(s)


def sdmd_server_set_graphs(s, on):
    _check(lib().sdmd_server_set_graphs(s, 1 if on else 0), "sdmd_server_set_graphs")


def sdmd_server_graph_stats(s):
    """(graphs built, graphs updated in place)"""
    b, u = _I64(), _I64()
    _check(lib().sdmd_server_graph_stats(s, ctypes.byref(b), ctypes.byref(u)), "sdmd_server_graph_stats")
    return b.value, u.value


def sdmd_server_autotune(s):
    _check(lib().sdmd_server_autotune(s), "sdmd_server_autotune")


def sdmd_server_reset_stats(s):
    _check(lib().sdmd_server_reset_stats(s), "sdmd_server_reset_stats")


def sdmd_server_clock_ms():
    return lib().sdmd_server_clock_ms()


def sdmd_amplitudes(h, b, stream=None, want_index=True):
    """Copy the mode amplitudes into `b` (r complex128 as 2r float64, host or
    device; may be None); returns the background mode index (or None)."""
    idx = _I32(-1)
    _check(lib().sdmd_amplitudes(h, ptr(b), ctypes.byref(idx) if want_index else None, stream_handle(stream)),
           "sdmd_amplitudes")
    return idx.value if want_index else None


def sdmd_reconstruct(h, t, what, out, stream=None):
    _check(lib().sdmd_reconstruct(h, int(t), int(what), ptr(out), stream_handle(stream)), "sdmd_reconstruct")


def sdmd_reconstruct_ex(h, t, what, tol, out, stream=None):
    _check(lib().sdmd_reconstruct_ex(h, int(t), int(what), float(tol), ptr(out), stream_handle(stream)),
           "sdmd_reconstruct_ex")


def sdmd_fourier_modes(h, r, idx=None, phi=None, cap=0, stream=None):
    """Compressed Phi-hat of the last sdmd_modes on a Fourier-sparse handle;
    returns the union size (cap = 0: count only)."""
    cnt = _I64()
    _check(lib().sdmd_fourier_modes(h, int(r), ptr(idx), ptr(phi), int(cap), ctypes.byref(cnt), stream_handle(stream)),
           "sdmd_fourier_modes")
    return cnt.value


def sdmd_autotune(h, stream=None):
    """Measure the Gram-row chunk schedules; returns (chunk_bytes, us per row)."""
    ch, us = _I64(), ctypes.c_double()
    _check(lib().sdmd_autotune(h, ctypes.byref(ch), ctypes.byref(us), stream_handle(stream)), "sdmd_autotune")
    return ch.value, us.value


def sdmd_pod_modes(h, r, U, stream=None):
    """U = X V Sigma^-1 (n x r float32, column-major) of the last sdmd_modes."""
    _check(lib().sdmd_pod_modes(h, int(r), ptr(U), stream_handle(stream)), "sdmd_pod_modes")


def sdmd_status(h, stream=None):
    return lib().sdmd_status(h, stream_handle(stream))


def sdmd_set_option(h, option, value):
    _check(lib().sdmd_set_option(h, int(option), int(value)), "sdmd_set_option")


def sdmd_trace(h, enable):
    _check(lib().sdmd_trace(h, 1 if enable else 0), "sdmd_trace")


def sdmd_trace_read(h, kernel):
    """(launches, total_ms) for kernel class `kernel` since the last read."""
    n = _I64()
    ms = ctypes.c_double()
    _check(lib().sdmd_trace_read(h, int(kernel), ctypes.byref(n), ctypes.byref(ms)), "sdmd_trace_read")
    return n.value, ms.value


MODES_PHASES = ["gather", "tridiagonalise", "bisection", "inverse_iteration", "back_transform",
                "atilde", "eig_atilde", "outputs"]


def sdmd_modes_phase_cycles(h, stream=None):
    """Per-phase SM cycles of the last FP64 modes kernel (dict)."""
    buf = (_I64 * 9)()
    _check(lib().sdmd_modes_phase_cycles(h, buf, 9, stream_handle(stream)), "sdmd_modes_phase_cycles")
    return {name: int(buf[i + 1] - buf[i]) for i, name in enumerate(MODES_PHASES)}


SDMD_GRAM_ROW_STATIC_MAX_C = 256


def sdmd_gram_row_static(dtype, X, ld, c, y, n, g, stream=None):
    """g[j] = <x_j, y> for j < c with no device allocation (see sdmd.h)."""
    _check(lib().sdmd_gram_row_static(int(dtype), ptr(X), int(ld), int(c), ptr(y), int(n), ptr(g),
                                      stream_handle(stream)), "sdmd_gram_row_static")


def sdmd_trace_times(h, kernel, cap=100000):
    """Individual traced durations (ms) of class `kernel` since the last read."""
    buf = (ctypes.c_double * cap)()
    cnt = _I32()
    _check(lib().sdmd_trace_times(h, int(kernel), buf, int(cap), ctypes.byref(cnt)), "sdmd_trace_times")
    return [buf[i] for i in range(cnt.value)]


def exported_symbols():
    """Names the binding expects the library to export."""
    return sorted(list(_SIGNATURES) + ["sdmd_last_error"])
