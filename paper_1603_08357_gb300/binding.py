"""Thin ctypes binding of libccl.so (include/ccl.h), same names as the C ABI.

Argument marshalling only: every step of the labelling runs in the library's
CUDA kernels. Device arrays may be given as torch CUDA tensors (int32, or
uint32/int32 for the bit words) or raw device addresses; host arrays as numpy
arrays or raw addresses; streams as torch streams, raw cudaStream_t values or
None (the current torch stream when torch is loaded, else the legacy default
stream). There is no CPU fallback: if the library cannot be loaded, importing
this module raises.
"""
from __future__ import annotations

import ctypes
import os
import sys

import numpy as np

from . import _build

CCL_OK = 0
CCL_ERR_INVALID_ARGUMENT = 1
CCL_ERR_INDEX_OUT_OF_RANGE = 2
CCL_ERR_ASYMMETRIC = 3
CCL_ERR_OUT_OF_MEMORY = 4
CCL_ERR_NONCONVERGED = 5
CCL_ERR_TIMEOUT = 6
CCL_ERR_REJECTED = 7
CCL_ERR_CUDA = 8
CCL_ERR_NOT_FOUND = 9

CCL_OPT_PRE_ANALYSIS = 0
CCL_OPT_BLOCK_THREADS = 1
CCL_OPT_USE_GRAPHS = 2
CCL_OPT_PROFILE = 3
CCL_OPT_CTAS_PER_SM = 4
CCL_OPT_LINK_MODE = 5
CCL_OPT_REFILL = 6
CCL_OPT_ANALYSIS_ORDER = 7
CCL_OPT_ITER_CAP = 8
CCL_OPT_REDUCE_WINDOW = 9
CCL_OPT_ANALYSIS_GROUP = 10
CCL_OPT_ANALYSIS_PARK = 11


class CclError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {ccl_status_string(status)} ({status})" if what else
                         f"{ccl_status_string(status)} ({status})")


class ccl_run_stats(ctypes.Structure):
    _fields_ = [("residual_pairs", ctypes.c_int64), ("n_sites", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("n_inst", ctypes.c_int32), ("used_graph", ctypes.c_int32),
                ("chase_loads", ctypes.c_int64), ("merge_atomics", ctypes.c_int64),
                ("reduce_iterations", ctypes.c_int64), ("pre_analysis", ctypes.c_int32),
                ("link_mode", ctypes.c_int32), ("refill", ctypes.c_int32), ("analysis_order", ctypes.c_int32),
                ("reduce_window", ctypes.c_int32), ("analysis_group", ctypes.c_int32),
                ("analysis_park", ctypes.c_int32)]


class ccl_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("n_streams", ctypes.c_int32),
                ("hbm_reserve", ctypes.c_int64), ("hbm_budget", ctypes.c_int64),
                ("max_batch", ctypes.c_int32), ("max_pending", ctypes.c_int32),
                ("host_staging_bytes", ctypes.c_int64)]


class ccl_request(ctypes.Structure):
    _fields_ = [("n_sites", ctypes.c_int32), ("pad_", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p),
                ("open_bits", ctypes.c_void_p)]


class ccl_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("sites_completed", ctypes.c_int64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("busy_seconds", ctypes.c_double), ("sites_per_second", ctypes.c_double),
                ("waiting", ctypes.c_int64), ("arena_misses", ctypes.c_int64),
                ("phase_p50_ms", ctypes.c_double * 4), ("phase_p99_ms", ctypes.c_double * 4)]


def _load() -> ctypes.CDLL:
    # CCL_LIB may name another build of the same ABI (e.g. a counting build)
    path = os.environ.get("CCL_LIB") or _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libccl.so is not built ({path}); run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    P, I32, I64, C = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int
    sigs = {
        "ccl_status_string": (ctypes.c_char_p, [C]),
        "ccl_version": (C, []),
        "ccl_context_create": (C, [ctypes.POINTER(P), C]),
        "ccl_context_destroy": (None, [P]),
        "ccl_set_option": (C, [P, C, I64]),
        "ccl_get_option": (C, [P, C, ctypes.POINTER(I64)]),
        "ccl_label": (C, [P, I32, I64, P, P, P, P, P]),
        "ccl_label_batched": (C, [P, I32, P, P, P, P, P, P, P]),
        "ccl_label_host": (C, [P, I32, I64, P, P, P, P, P]),
        "ccl_label_batched_host": (C, [P, I32, P, P, P, P, P, P, P]),
        "ccl_label_random": (C, [P, I32, I64, P, P, ctypes.c_uint64, ctypes.c_double, P, P]),
        "ccl_label_dense": (C, [P, I32, I32, P, P, P, P]),
        "ccl_label_dense_random": (C, [P, I32, I32, P, ctypes.c_uint64, ctypes.c_double, P, P]),
        "ccl_label_noalloc": (C, [I32, I64, P, P, P, P, P]),
        "ccl_reserve": (C, [P, I64, I64, I64]),
        "ccl_relabel": (C, [P, I32, P, P, P, P, P]),
        "ccl_spanning": (C, [P, I32, P, P, I32, P, I32, P, P]),
        "ccl_largest_cluster": (C, [P, I32, P, P, P]),
        "ccl_sync": (C, [P, P, I64]),
        "ccl_validate": (C, [P, I32, I64, P, P, P, P]),
        "ccl_get_stats": (C, [P, ctypes.POINTER(ccl_run_stats)]),
        "ccl_get_step_times": (C, [P, ctypes.POINTER(ctypes.c_float), I32]),
        "ccl_autotune": (C, [P, I32, I64, P, P, P, P, P, ctypes.POINTER(ctypes.c_float)]),
        "ccl_autotune_batched": (C, [P, I32, P, P, P, P, P, P, P, ctypes.POINTER(ctypes.c_float)]),
        "ccl_server_create": (C, [ctypes.POINTER(P), ctypes.POINTER(ccl_server_config)]),
        "ccl_server_submit": (C, [P, ctypes.POINTER(ccl_request), ctypes.POINTER(ctypes.c_uint64)]),
        "ccl_server_submit_nocopy": (C, [P, ctypes.POINTER(ccl_request), ctypes.POINTER(ctypes.c_uint64)]),
        "ccl_server_wait": (C, [P, ctypes.c_uint64, P, I64]),
        "ccl_server_stats_get": (C, [P, ctypes.POINTER(ccl_server_stats)]),
        "ccl_server_destroy": (None, [P]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()
LIB_PATH = os.environ.get("CCL_LIB") or _build.LIB


# ----------------------------------------------------------------------------
# marshalling helpers

def _dev_ptr(x, name: str, dtypes=None):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    torch = sys.modules.get("torch")
    if torch is not None and isinstance(x, torch.Tensor):
        if not x.is_cuda:
            raise TypeError(f"{name}: expected a CUDA tensor")
        if not x.is_contiguous():
            raise TypeError(f"{name}: tensor must be contiguous")
        if dtypes is not None and x.dtype not in dtypes:
            raise TypeError(f"{name}: dtype {x.dtype} not in {dtypes}")
        return x.data_ptr()
    raise TypeError(f"{name}: expected a torch CUDA tensor or a device address")


def _host_ptr(x, name: str, dtype=None):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    torch = sys.modules.get("torch")
    if torch is not None and isinstance(x, torch.Tensor):
        if x.is_cuda or not x.is_contiguous():
            raise TypeError(f"{name}: expected a contiguous host tensor")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise TypeError(f"{name}: array must be C-contiguous")
        if dtype is not None and x.dtype != dtype:
            raise TypeError(f"{name}: dtype {x.dtype} != {dtype}")
        return x.ctypes.data
    raise TypeError(f"{name}: expected a numpy array, host tensor or address")


def _stream(s):
    if s is None:
        torch = sys.modules.get("torch")
        if torch is not None and torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _i32():
    import torch
    return (torch.int32,)


def _bits_dtypes():
    import torch
    return tuple(d for d in (torch.int32, getattr(torch, "uint32", None)) if d is not None)


class Context:
    """Owns a ccl_context handle; destroyed with the object."""

    def __init__(self, handle: int, device: int):
        self.handle = handle
        self.device = device

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h:
            _lib.ccl_context_destroy(h)

    @property
    def _as_parameter_(self):
        return ctypes.c_void_p(self.handle)


class Server:
    def __init__(self, handle: int):
        self.handle = handle

    def close(self):
        h, self.handle = self.handle, None
        if h:
            _lib.ccl_server_destroy(h)

    def __del__(self):
        if getattr(self, "handle", None):
            self.close()

    @property
    def _as_parameter_(self):
        return ctypes.c_void_p(self.handle)


def check(status: int, what: str = "") -> None:
    if status != CCL_OK:
        raise CclError(status, what)


# ----------------------------------------------------------------------------
# the C ABI, same names

def ccl_status_string(status: int) -> str:
    return _lib.ccl_status_string(int(status)).decode()


def ccl_version() -> int:
    return int(_lib.ccl_version())


def ccl_context_create(device: int = 0) -> Context:
    h = ctypes.c_void_p()
    check(_lib.ccl_context_create(ctypes.byref(h), int(device)), "ccl_context_create")
    return Context(h.value, device)


def ccl_context_destroy(ctx: Context) -> None:
    h, ctx.handle = ctx.handle, None
    if h:
        _lib.ccl_context_destroy(h)


def ccl_set_option(ctx, option: int, value: int) -> int:
    return _lib.ccl_set_option(ctx, int(option), int(value))


def ccl_get_option(ctx, option: int) -> int:
    v = ctypes.c_int64()
    check(_lib.ccl_get_option(ctx, int(option), ctypes.byref(v)), "ccl_get_option")
    return int(v.value)


def ccl_label(ctx, n_sites: int, nnz: int, row_ptr, col_idx, open_bits, labels, stream=None) -> int:
    return _lib.ccl_label(ctx, int(n_sites), int(nnz), _dev_ptr(row_ptr, "row_ptr", _i32()),
                          _dev_ptr(col_idx, "col_idx", _i32()),
                          _dev_ptr(open_bits, "open_bits", _bits_dtypes()),
                          _dev_ptr(labels, "labels", _i32()), _stream(stream))


def ccl_label_batched(ctx, n_inst: int, site_off, ent_off, row_ptr, col_idx, open_bits, labels,
                      stream=None) -> int:
    so = np.ascontiguousarray(site_off, dtype=np.int64)
    eo = np.ascontiguousarray(ent_off, dtype=np.int64)
    if so.size != n_inst + 1 or eo.size != n_inst + 1:
        return CCL_ERR_INVALID_ARGUMENT
    return _lib.ccl_label_batched(ctx, int(n_inst), so.ctypes.data, eo.ctypes.data,
                                  _dev_ptr(row_ptr, "row_ptr", _i32()),
                                  _dev_ptr(col_idx, "col_idx", _i32()),
                                  _dev_ptr(open_bits, "open_bits", _bits_dtypes()),
                                  _dev_ptr(labels, "labels", _i32()), _stream(stream))


def ccl_label_random(ctx, n_sites: int, nnz: int, row_ptr, col_idx, seed: int, p: float, labels,
                     stream=None) -> int:
    return _lib.ccl_label_random(ctx, int(n_sites), int(nnz), _dev_ptr(row_ptr, "row_ptr", _i32()),
                                 _dev_ptr(col_idx, "col_idx", _i32()), ctypes.c_uint64(seed & (2**64 - 1)),
                                 float(p), _dev_ptr(labels, "labels", _i32()), _stream(stream))


CCL_DENSE_MAX_WIDTH = 4096
CCL_MAX_SITES = 2147479551          # most sites of one instance (2^31 - 4097)


def ccl_label_dense(ctx, n_sites: int, width: int, nn, open_bits, labels, stream=None) -> int:
    return _lib.ccl_label_dense(ctx, int(n_sites), int(width), _dev_ptr(nn, "nn", _i32()),
                                _dev_ptr(open_bits, "open_bits", _bits_dtypes()),
                                _dev_ptr(labels, "labels", _i32()), _stream(stream))


def ccl_label_dense_random(ctx, n_sites: int, width: int, nn, seed: int, p: float, labels,
                           stream=None) -> int:
    return _lib.ccl_label_dense_random(ctx, int(n_sites), int(width), _dev_ptr(nn, "nn", _i32()),
                                       ctypes.c_uint64(seed & (2**64 - 1)), float(p),
                                       _dev_ptr(labels, "labels", _i32()), _stream(stream))


def ccl_label_host(ctx, n_sites: int, nnz: int, row_ptr, col_idx, open_bits, labels,
                   stream=None) -> int:
    return _lib.ccl_label_host(ctx, int(n_sites), int(nnz), _host_ptr(row_ptr, "row_ptr", np.int32),
                               _host_ptr(col_idx, "col_idx", np.int32),
                               _host_ptr(open_bits, "open_bits", np.uint32),
                               _host_ptr(labels, "labels", np.int32), _stream(stream))


def ccl_label_batched_host(ctx, n_inst: int, site_off, ent_off, row_ptr, col_idx, open_bits, labels,
                           stream=None) -> int:
    """ccl_label_batched on host arrays; synchronous (see ccl.h)."""
    so = np.ascontiguousarray(site_off, dtype=np.int64)
    eo = np.ascontiguousarray(ent_off, dtype=np.int64)
    if so.size != n_inst + 1 or eo.size != n_inst + 1:
        return CCL_ERR_INVALID_ARGUMENT
    return _lib.ccl_label_batched_host(ctx, int(n_inst), so.ctypes.data, eo.ctypes.data,
                                       _host_ptr(row_ptr, "row_ptr", np.int32),
                                       _host_ptr(col_idx, "col_idx", np.int32),
                                       _host_ptr(open_bits, "open_bits", np.uint32),
                                       _host_ptr(labels, "labels", np.int32), _stream(stream))


def ccl_label_noalloc(n_sites: int, nnz: int, row_ptr, col_idx, open_bits, labels, stream=None) -> int:
    """Allocation-free, synchronous single-instance labelling (see ccl.h)."""
    return _lib.ccl_label_noalloc(int(n_sites), int(nnz), _dev_ptr(row_ptr, "row_ptr", _i32()),
                                  _dev_ptr(col_idx, "col_idx", _i32()),
                                  _dev_ptr(open_bits, "open_bits", _bits_dtypes()),
                                  _dev_ptr(labels, "labels", _i32()), _stream(stream))


def ccl_reserve(ctx, n_sites: int, nnz: int, n_chunks: int = 0) -> int:
    return _lib.ccl_reserve(ctx, int(n_sites), int(nnz), int(n_chunks))


def ccl_relabel(ctx, n: int, labels, seq, n_clusters, sizes=None, stream=None) -> int:
    return _lib.ccl_relabel(ctx, int(n), _dev_ptr(labels, "labels", _i32()), _dev_ptr(seq, "seq", _i32()),
                            _dev_ptr(n_clusters, "n_clusters", _i32()), _dev_ptr(sizes, "sizes", _i32()),
                            _stream(stream))


def ccl_spanning(ctx, n: int, labels, top, n_top: int, bottom, n_bottom: int, result, stream=None) -> int:
    return _lib.ccl_spanning(ctx, int(n), _dev_ptr(labels, "labels", _i32()), _dev_ptr(top, "top", _i32()),
                             int(n_top), _dev_ptr(bottom, "bottom", _i32()), int(n_bottom),
                             _dev_ptr(result, "result", _i32()), _stream(stream))


def ccl_largest_cluster(ctx, n: int, labels, result, stream=None) -> int:
    """result: DEVICE int32[2] <- (size, label) of the largest cluster."""
    return _lib.ccl_largest_cluster(ctx, int(n), _dev_ptr(labels, "labels", _i32()),
                                    _dev_ptr(result, "result", _i32()), _stream(stream))


def ccl_sync(ctx, stream=None, timeout_ms: int = -1) -> int:
    return _lib.ccl_sync(ctx, _stream(stream), int(timeout_ms))


def ccl_validate(ctx, n_sites: int, nnz: int, row_ptr, col_idx, open_bits, stream=None) -> int:
    return _lib.ccl_validate(ctx, int(n_sites), int(nnz), _dev_ptr(row_ptr, "row_ptr", _i32()),
                             _dev_ptr(col_idx, "col_idx", _i32()),
                             _dev_ptr(open_bits, "open_bits", _bits_dtypes()), _stream(stream))


def ccl_get_stats(ctx) -> ccl_run_stats:
    st = ccl_run_stats()
    check(_lib.ccl_get_stats(ctx, ctypes.byref(st)), "ccl_get_stats")
    return st


def ccl_get_step_times(ctx) -> list:
    """[init, analysis (ii), reduction (iii), analysis (iv)] mean ms, then the call count."""
    arr = (ctypes.c_float * 5)()
    check(_lib.ccl_get_step_times(ctx, arr, 5), "ccl_get_step_times")
    return [float(v) for v in arr]


def ccl_autotune(ctx, n_sites: int, nnz: int, row_ptr, col_idx, open_bits, labels, stream=None):
    best = ctypes.c_float(0)
    st = _lib.ccl_autotune(ctx, int(n_sites), int(nnz), _dev_ptr(row_ptr, "row_ptr", _i32()),
                           _dev_ptr(col_idx, "col_idx", _i32()),
                           _dev_ptr(open_bits, "open_bits", _bits_dtypes()),
                           _dev_ptr(labels, "labels", _i32()), _stream(stream), ctypes.byref(best))
    return st, float(best.value)


def ccl_autotune_batched(ctx, n_inst: int, site_off, ent_off, row_ptr, col_idx, open_bits, labels,
                         stream=None):
    so = np.ascontiguousarray(site_off, dtype=np.int64)
    eo = np.ascontiguousarray(ent_off, dtype=np.int64)
    if so.size != n_inst + 1 or eo.size != n_inst + 1:
        return CCL_ERR_INVALID_ARGUMENT, 0.0
    best = ctypes.c_float(0)
    st = _lib.ccl_autotune_batched(ctx, int(n_inst), so.ctypes.data, eo.ctypes.data,
                                   _dev_ptr(row_ptr, "row_ptr", _i32()), _dev_ptr(col_idx, "col_idx", _i32()),
                                   _dev_ptr(open_bits, "open_bits", _bits_dtypes()),
                                   _dev_ptr(labels, "labels", _i32()), _stream(stream), ctypes.byref(best))
    return st, float(best.value)


def ccl_server_create(device: int = 0, n_streams: int = 2, hbm_reserve: int = 0, hbm_budget: int = 0,
                      max_batch: int = 0, max_pending: int = 0, host_staging_bytes: int = 0) -> Server:
    cfg = ccl_server_config(int(device), int(n_streams), int(hbm_reserve), int(hbm_budget),
                            int(max_batch), int(max_pending), int(host_staging_bytes))
    h = ctypes.c_void_p()
    check(_lib.ccl_server_create(ctypes.byref(h), ctypes.byref(cfg)), "ccl_server_create")
    return Server(h.value)


def ccl_server_submit(srv, n_sites: int, nnz: int, row_ptr, col_idx, open_bits):
    """Returns (status, ticket). Host arrays are copied before it returns."""
    req = ccl_request(int(n_sites), 0, int(nnz), _host_ptr(row_ptr, "row_ptr", np.int32),
                      _host_ptr(col_idx, "col_idx", np.int32),
                      _host_ptr(open_bits, "open_bits", np.uint32))
    t = ctypes.c_uint64(0)
    st = _lib.ccl_server_submit(srv, ctypes.byref(req), ctypes.byref(t))
    return st, int(t.value)


def ccl_server_submit_nocopy(srv, n_sites: int, nnz: int, row_ptr, col_idx, open_bits):
    """Returns (status, ticket). The host arrays are NOT copied: keep them alive
    and unchanged until ccl_server_wait has returned for the ticket."""
    req = ccl_request(int(n_sites), 0, int(nnz), _host_ptr(row_ptr, "row_ptr", np.int32),
                      _host_ptr(col_idx, "col_idx", np.int32),
                      _host_ptr(open_bits, "open_bits", np.uint32))
    t = ctypes.c_uint64(0)
    st = _lib.ccl_server_submit_nocopy(srv, ctypes.byref(req), ctypes.byref(t))
    return st, int(t.value)


def ccl_server_wait(srv, ticket: int, labels_host, timeout_ms: int = -1) -> int:
    return _lib.ccl_server_wait(srv, ctypes.c_uint64(ticket), _host_ptr(labels_host, "labels", np.int32),
                                int(timeout_ms))


def ccl_server_stats_get(srv) -> ccl_server_stats:
    st = ccl_server_stats()
    check(_lib.ccl_server_stats_get(srv, ctypes.byref(st)), "ccl_server_stats_get")
    return st


def ccl_server_destroy(srv) -> None:
    srv.close()
