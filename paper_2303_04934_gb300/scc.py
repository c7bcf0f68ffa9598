"""Thin Python binding of the C ABI in ``include/scc.h``, ``include/scc_batch.h``,
``include/scc_serve.h`` and ``include/scc_debug.h``.

Argument marshalling only: every step runs in the CUDA library
``_lib/libscc_gb300.so``. Arrays may be CUDA torch tensors (device pointers are
passed) or numpy arrays / CPU tensors (host pointers are passed; the library
copies). Streams are ``torch.cuda.Stream`` objects or None (torch's current
stream). There is no CPU fallback: if the library is missing, loading fails.

The function names are those of the C ABI.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SCC_OK = 0
SCC_ERR_INVALID_ARG = -1
SCC_ERR_OOM = -2
SCC_ERR_CUDA = -3
SCC_ERR_TIMEOUT = -4
SCC_ERR_CAPACITY = -5
SCC_ERR_INTERNAL = -6

#: every symbol the headers declare (checked by tests/test_abi_symbols.py)
EXPORTED = [
    "scc_error_string", "scc_config_default", "scc_graph_create", "scc_graph_destroy", "scc_set_config",
    "scc_run", "reach_multi", "reach_multi_noalloc", "scc_get_stats", "cc_run", "cc_get_stats",
    "le_lists_run", "le_lists_get", "le_get_stats",
    "scc_graph_info", "scc_debug_csr", "scc_debug_trim", "scc_debug_pivot_order", "scc_debug_single_reach",
    "scc_debug_multi_reach", "scc_debug_reach_multi_wide", "scc_debug_hashbag", "scc_debug_pair_table", "scc_debug_launch_count",
    "scc_debug_barrier_timeout", "scc_debug_le_lists",
    "scc_batch_config_default", "scc_batch_create", "scc_batch_destroy", "scc_batch_set_config",
    "scc_batch_get_config", "scc_batch_run", "scc_batch_autotune", "scc_batch_get_stats",
    "scc_debug_batch_times", "scc_debug_batch_groups", "scc_debug_serve_admission", "scc_debug_serve_unit",
    "scc_server_config_default", "scc_server_create", "scc_server_destroy", "scc_server_add_graph",
    "scc_server_remove_graph", "scc_server_submit_scc", "scc_server_submit_reach", "scc_server_wait",
    "scc_server_drain", "scc_server_get_stats", "scc_server_reset_stats",
]


class scc_config(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_int32), ("beta", ctypes.c_double), ("lambda_", ctypes.c_int32),
                ("sigma", ctypes.c_int32), ("block", ctypes.c_int32), ("seeds", ctypes.c_int32),
                ("dense", ctypes.c_int32), ("seed", ctypes.c_uint64), ("ldd_beta", ctypes.c_double)]


class scc_stats(ctypes.Structure):
    _fields_ = [("n_trimmed", ctypes.c_int32), ("first_scc_size", ctypes.c_int32), ("batches", ctypes.c_int32),
                ("search_rounds", ctypes.c_int32), ("pairs", ctypes.c_int64), ("table_resizes", ctypes.c_int32),
                ("engine_launches", ctypes.c_int32), ("ms_trim", ctypes.c_double), ("ms_first_scc", ctypes.c_double),
                ("ms_multi_search", ctypes.c_double), ("ms_resize", ctypes.c_double), ("ms_label", ctypes.c_double),
                ("ms_engine", ctypes.c_double), ("engine_arcs", ctypes.c_int64), ("engine_items", ctypes.c_int64),
                ("engine_inserted", ctypes.c_int64), ("ms_create", ctypes.c_double),
                ("ms_transpose_hist", ctypes.c_double), ("ms_transpose_part", ctypes.c_double),
                ("ms_transpose_rows", ctypes.c_double), ("n_class_trimmed", ctypes.c_int32),
                ("class_trim_passes", ctypes.c_int32), ("ms_class_trim", ctypes.c_double),
                ("multi_launches", ctypes.c_int32), ("multi_arcs", ctypes.c_int64), ("multi_items", ctypes.c_int64),
                ("tau", ctypes.c_int32), ("ms_transpose_split", ctypes.c_double),
                ("multi_active_sum", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class scc_cc_stats(ctypes.Structure):
    _fields_ = [("components", ctypes.c_int32), ("clusters", ctypes.c_int32), ("ldd_rounds", ctypes.c_int32),
                ("ldd_batches", ctypes.c_int32), ("ldd_arcs", ctypes.c_int64), ("cross_arcs", ctypes.c_int64),
                ("ms_sym", ctypes.c_double), ("ms_ldd", ctypes.c_double), ("ms_union", ctypes.c_double),
                ("ms_label", ctypes.c_double), ("ms_total", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class scc_le_stats(ctypes.Structure):
    _fields_ = [("entries", ctypes.c_int64), ("candidates", ctypes.c_int64), ("arcs", ctypes.c_int64),
                ("levels", ctypes.c_int32), ("launches", ctypes.c_int32), ("ms_total", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class scc_batch_config(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_int32), ("block", ctypes.c_int32), ("lambda_", ctypes.c_int32),
                ("sigma", ctypes.c_int32), ("seeds", ctypes.c_int32), ("beta", ctypes.c_double),
                ("blocks_per_sm", ctypes.c_int32), ("seed", ctypes.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class scc_batch_stats(ctypes.Structure):
    _fields_ = [("graphs", ctypes.c_int32), ("vertices", ctypes.c_int64), ("arcs", ctypes.c_int64),
                ("max_vertices", ctypes.c_int32), ("max_arcs", ctypes.c_int64), ("blocks", ctypes.c_int32),
                ("workspace_bytes", ctypes.c_int64), ("ms_last_run", ctypes.c_double), ("captures", ctypes.c_int32),
                ("replays", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class scc_server_config(ctypes.Structure):
    _fields_ = [("mem_cap_bytes", ctypes.c_int64), ("batch_vertices", ctypes.c_int32),
                ("batch_graphs", ctypes.c_int32), ("merge_reach", ctypes.c_int32), ("prefetch", ctypes.c_int32),
                ("max_bypass_ms", ctypes.c_double), ("batch_min", ctypes.c_int32)]


class scc_server_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in (
        "submitted", "completed", "failed", "scc_requests", "reach_requests", "units", "batched_launches",
        "batched_graphs", "plain_scc", "reach_launches", "reach_shared", "mem_in_use", "mem_peak", "mem_cap")] + [
        ("max_admitted", ctypes.c_int32), ("resident_graphs", ctypes.c_int32)] + [
        (f, ctypes.c_double) for f in ("p50_ms", "p99_ms", "scc_p50_ms", "scc_p99_ms", "reach_p50_ms",
                                        "reach_p99_ms", "busy_reach_ms", "busy_batched_ms", "busy_plain_ms")]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SccError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {error_string(code)} ({code})")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.SO_PATH


def load() -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.SO_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: run __graft_entry__.build() "
                           "(or python -m paper_2303_04934_gb300.build) first")
    lib = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    P = ctypes.POINTER
    sig = {
        "scc_error_string": ([ctypes.c_int], ctypes.c_char_p),
        "scc_config_default": ([P(scc_config)], ctypes.c_int),
        "scc_graph_create": ([i32, i64, vp, vp, vp, P(vp)], ctypes.c_int),
        "scc_graph_destroy": ([vp], ctypes.c_int),
        "scc_set_config": ([vp, P(scc_config)], ctypes.c_int),
        "scc_run": ([vp, vp, vp], ctypes.c_int),
        "reach_multi": ([vp, vp, i32, i32, vp, vp], ctypes.c_int),
        "reach_multi_noalloc": ([vp, vp, i32, i32, vp, vp], ctypes.c_int),
        "scc_get_stats": ([vp, P(scc_stats)], ctypes.c_int),
        "cc_run": ([vp, vp, vp], ctypes.c_int),
        "cc_get_stats": ([vp, P(scc_cc_stats)], ctypes.c_int),
        "le_lists_run": ([vp, P(i64), vp], ctypes.c_int),
        "le_lists_get": ([vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "le_get_stats": ([vp, P(scc_le_stats)], ctypes.c_int),
        "scc_graph_info": ([vp, P(i32), P(i64), P(i64)], ctypes.c_int),
        "scc_debug_csr": ([vp, i32, vp, vp, vp], ctypes.c_int),
        "scc_debug_trim": ([vp, vp, vp], ctypes.c_int),
        "scc_debug_pivot_order": ([vp, vp, P(i32), vp], ctypes.c_int),
        "scc_debug_single_reach": ([vp, vp, i32, i32, vp, vp], ctypes.c_int),
        "scc_debug_multi_reach": ([vp, vp, vp, i32, i32, vp, i64, P(i64), i64, vp], ctypes.c_int),
        "scc_debug_reach_multi_wide": ([vp, vp, i32, i32, vp, vp], ctypes.c_int),
        "scc_debug_hashbag": ([vp, i64, i32, i32, vp, P(i64), P(i32), vp], ctypes.c_int),
        "scc_debug_pair_table": ([vp, i64, i64, vp, P(i64), P(i32), vp], ctypes.c_int),
        "scc_debug_launch_count": ([], ctypes.c_int64),
        "scc_debug_barrier_timeout": ([i32, i64, P(i32), vp], ctypes.c_int),
        "scc_debug_le_lists": ([vp, i64, i64, P(i64), vp], ctypes.c_int),
        "scc_batch_config_default": ([P(scc_batch_config)], ctypes.c_int),
        "scc_batch_create": ([i32, vp, vp, vp, vp, vp, P(vp)], ctypes.c_int),
        "scc_batch_destroy": ([vp], ctypes.c_int),
        "scc_batch_set_config": ([vp, P(scc_batch_config)], ctypes.c_int),
        "scc_batch_get_config": ([vp, P(scc_batch_config)], ctypes.c_int),
        "scc_batch_run": ([vp, vp, vp], ctypes.c_int),
        "scc_batch_autotune": ([vp, i32, vp, P(scc_batch_config), P(ctypes.c_double)], ctypes.c_int),
        "scc_batch_get_stats": ([vp, P(scc_batch_stats)], ctypes.c_int),
        "scc_debug_batch_times": ([vp, vp], ctypes.c_int),
        "scc_debug_batch_groups": ([i32, vp, vp, i64, i64, vp, P(i32)], ctypes.c_int),
        "scc_debug_serve_admission": ([i32, vp, vp, i64, i64, ctypes.c_double, vp, P(i32)], ctypes.c_int),
        "scc_debug_serve_unit": ([i32, vp, vp, vp, vp, vp, i32, i32, i32, vp, P(i32)], ctypes.c_int),
        "scc_server_config_default": ([P(scc_server_config)], ctypes.c_int),
        "scc_server_create": ([P(scc_server_config), P(vp)], ctypes.c_int),
        "scc_server_destroy": ([vp], ctypes.c_int),
        "scc_server_add_graph": ([vp, i32, i64, vp, vp, P(i32)], ctypes.c_int),
        "scc_server_remove_graph": ([vp, i32], ctypes.c_int),
        "scc_server_submit_scc": ([vp, i32, i64, vp, vp, vp, P(i64)], ctypes.c_int),
        "scc_server_submit_reach": ([vp, i32, vp, i32, i32, vp, P(i64)], ctypes.c_int),
        "scc_server_wait": ([vp, i64, P(i32), P(ctypes.c_double)], ctypes.c_int),
        "scc_server_drain": ([vp], ctypes.c_int),
        "scc_server_get_stats": ([vp, P(scc_server_stats)], ctypes.c_int),
        "scc_server_reset_stats": ([vp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def error_string(code: int) -> str:
    try:
        return load().scc_error_string(code).decode()
    except Exception:  # pragma: no cover - only when the library cannot load
        return f"error {code}"


def _check(rc: int, what: str):
    if rc != SCC_OK:
        raise SccError(rc, what)


def _ptr(a):
    """Raw pointer of a torch tensor (device or host) or a numpy array."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


I32 = ("int32",)
I64 = ("int64",)
W64 = ("uint64", "int64")  # 64-bit reachability masks


def _elements(a):
    return int(a.size) if isinstance(a, np.ndarray) else int(a.numel())


def _arr(a, what: str, types, count: int):
    """_ptr of an argument the C ABI reads or writes as `count` elements of one
    of `types`: a wrong element type or a shorter array raises SccError
    (SCC_ERR_INVALID_ARG) here, before the library could misread it or write
    past its end."""
    if a is None:
        if count > 0:
            raise SccError(SCC_ERR_INVALID_ARG, f"{what}: missing")
        return None
    name = a.dtype.name if isinstance(a, np.ndarray) else str(getattr(a, "dtype", "")).replace("torch.", "")
    if name not in types:
        raise SccError(SCC_ERR_INVALID_ARG, f"{what}: elements of type {name}, expected {' or '.join(types)}")
    if _elements(a) < count:
        raise SccError(SCC_ERR_INVALID_ARG, f"{what}: {_elements(a)} elements, {count} needed")
    return _ptr(a)


def _stream(stream):
    if stream is None:
        import torch
        if not torch.cuda.is_available():
            return None
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


# ------------------------------------------------------------------- config --
def scc_config_default() -> scc_config:
    c = scc_config()
    _check(load().scc_config_default(ctypes.byref(c)), "scc_config_default")
    return c


# ------------------------------------------------------------------- graphs --
def scc_graph_create(n: int, m: int, offsets, targets, stream=None) -> int:
    h = ctypes.c_void_p()
    what = "scc_graph_create"
    po = _arr(offsets, what + " offsets", I32, max(n, 0) + 1)
    pt = _arr(targets, what + " targets", I32, max(m, 0))
    _check(load().scc_graph_create(n, m, po, pt, _stream(stream), ctypes.byref(h)), what)
    return h.value


def scc_graph_destroy(h) -> None:
    _check(load().scc_graph_destroy(h), "scc_graph_destroy")


def scc_set_config(h, cfg: scc_config) -> None:
    _check(load().scc_set_config(h, ctypes.byref(cfg)), "scc_set_config")


def scc_run(h, labels_out, stream=None) -> None:
    n = scc_graph_info(h)[0]
    _check(load().scc_run(h, _arr(labels_out, "scc_run labels_out", I32, n), _stream(stream)), "scc_run")


def cc_run(h, labels_out, stream=None) -> None:
    n = scc_graph_info(h)[0]
    _check(load().cc_run(h, _arr(labels_out, "cc_run labels_out", I32, n), _stream(stream)), "cc_run")


def cc_get_stats(h) -> dict:
    s = scc_cc_stats()
    _check(load().cc_get_stats(h, ctypes.byref(s)), "cc_get_stats")
    return s.as_dict()


def le_lists_run(h, stream=None) -> int:
    """Computes the handle's least-element lists; returns the number of entries."""
    total = ctypes.c_int64()
    _check(load().le_lists_run(h, ctypes.byref(total), _stream(stream)), "le_lists_run")
    return total.value


def le_lists_get(h, order, le_off, le_src, le_dist, total: int, stream=None) -> None:
    n = scc_graph_info(h)[0]
    what = "le_lists_get"
    _check(load().le_lists_get(h, _arr(order, what + " order", I32, n), _arr(le_off, what + " le_off", I64, n + 1),
                               _arr(le_src, what + " le_src", I32, total), _arr(le_dist, what + " le_dist", I32, total),
                               _stream(stream)), what)


def scc_debug_le_lists(h, init_cap: int, init_log: int, stream=None) -> int:
    total = ctypes.c_int64()
    _check(load().scc_debug_le_lists(h, init_cap, init_log, ctypes.byref(total), _stream(stream)),
           "scc_debug_le_lists")
    return total.value


def le_get_stats(h) -> dict:
    s = scc_le_stats()
    _check(load().le_get_stats(h, ctypes.byref(s)), "le_get_stats")
    return s.as_dict()


def reach_multi(h, sources, k: int, dir: int, out, stream=None) -> None:
    n = scc_graph_info(h)[0]
    ps = _arr(sources, "reach_multi sources", I32, k)
    _check(load().reach_multi(h, ps, k, dir, _arr(out, "reach_multi out", W64, n), _stream(stream)), "reach_multi")


def reach_multi_noalloc(h, sources, k: int, dir: int, out, stream=None) -> None:
    """reach_multi for callers that cannot allocate: device buffers only, working
    memory from the library's fixed 32 MiB device array (see include/scc.h)."""
    n = scc_graph_info(h)[0]
    ps = _arr(sources, "reach_multi_noalloc sources", I32, k)
    _check(load().reach_multi_noalloc(h, ps, k, dir, _arr(out, "reach_multi_noalloc out", W64, n), _stream(stream)),
           "reach_multi_noalloc")


def scc_get_stats(h) -> dict:
    s = scc_stats()
    _check(load().scc_get_stats(h, ctypes.byref(s)), "scc_get_stats")
    return s.as_dict()


# ------------------------------------------------------------------ batches --
def scc_batch_config_default() -> scc_batch_config:
    c = scc_batch_config()
    _check(load().scc_batch_config_default(ctypes.byref(c)), "scc_batch_config_default")
    return c


def scc_batch_create(G: int, vbase, ebase, offsets, targets, stream=None) -> int:
    h = ctypes.c_void_p()
    what = "scc_batch_create"
    pv = _arr(vbase, what + " vbase", I64, max(G, 0) + 1)
    pe = _arr(ebase, what + " ebase", I64, max(G, 0) + 1)
    po = _arr(offsets, what + " offsets", I32, 0)
    pt = _arr(targets, what + " targets", I32, 0)
    _check(load().scc_batch_create(G, pv, pe, po, pt, _stream(stream), ctypes.byref(h)), what)
    return h.value


def scc_batch_destroy(h) -> None:
    _check(load().scc_batch_destroy(h), "scc_batch_destroy")


def scc_batch_set_config(h, cfg: scc_batch_config) -> None:
    _check(load().scc_batch_set_config(h, ctypes.byref(cfg)), "scc_batch_set_config")


def scc_batch_get_config(h) -> scc_batch_config:
    c = scc_batch_config()
    _check(load().scc_batch_get_config(h, ctypes.byref(c)), "scc_batch_get_config")
    return c


def scc_batch_run(h, labels_out, stream=None) -> None:
    nv = scc_batch_get_stats(h)["vertices"]
    _check(load().scc_batch_run(h, _arr(labels_out, "scc_batch_run labels_out", I32, nv), _stream(stream)),
           "scc_batch_run")


def scc_batch_autotune(h, sample: int = 0, stream=None):
    best, ms = scc_batch_config(), ctypes.c_double()
    _check(load().scc_batch_autotune(h, sample, _stream(stream), ctypes.byref(best), ctypes.byref(ms)),
           "scc_batch_autotune")
    return best, ms.value


def scc_batch_get_stats(h) -> dict:
    s = scc_batch_stats()
    _check(load().scc_batch_get_stats(h, ctypes.byref(s)), "scc_batch_get_stats")
    return s.as_dict()


def scc_debug_batch_times(h, G: int) -> np.ndarray:
    """(G, 11) uint64 per graph of the last run: globaltimer ns at its start and
    after the transpose, single-pivot steps, class trimming, batches and
    labels; block; batch rounds, pair searches, reruns, batches."""
    out = np.zeros(11 * max(G, 1), np.uint64)
    _check(load().scc_debug_batch_times(h, _ptr(out)), "scc_debug_batch_times")
    return out[:11 * G].reshape(G, 11)


def scc_debug_batch_groups(vbase, ebase, max_vertices: int = 1 << 24, max_arcs: int = 1 << 27) -> list:
    """Groups [(g0, g1), ...] of consecutive graphs for the G^T passes of a
    batched run (host only)."""
    vb = np.ascontiguousarray(vbase, dtype=np.int64)
    eb = np.ascontiguousarray(ebase, dtype=np.int64)
    G = len(vb) - 1
    out = np.zeros(2 * max(G, 1), np.int32)
    ng = ctypes.c_int32()
    _check(load().scc_debug_batch_groups(G, _ptr(vb), _ptr(eb), max_vertices, max_arcs, _ptr(out), ctypes.byref(ng)),
           "scc_debug_batch_groups")
    return [(int(out[2 * k]), int(out[2 * k + 1])) for k in range(ng.value)]


def scc_debug_serve_admission(need, waited_ms, in_use: int, cap: int, max_bypass_ms: float) -> list:
    """Indices of the pending requests (arrival order) one admission pass of the
    server admits (host only)."""
    nd = np.ascontiguousarray(need, dtype=np.int64)
    wt = np.ascontiguousarray(waited_ms, dtype=np.float64)
    if len(nd) != len(wt):
        raise ValueError("need and waited_ms differ in length")
    out = np.zeros(max(len(nd), 1), np.int32)
    na = ctypes.c_int32()
    _check(load().scc_debug_serve_admission(len(nd), _ptr(nd), _ptr(wt), in_use, cap, max_bypass_ms, _ptr(out),
                                            ctypes.byref(na)), "scc_debug_serve_admission")
    return out[:na.value].tolist()


def scc_debug_serve_unit(kind, small, graph, dir, nsrc, merge_reach: bool = True, batch_graphs: int = 512,
                         batch_min: int = 1) -> list:
    """Indices of the admitted requests (arrival order) that join the unit of
    the oldest one (host only)."""
    cols = [np.ascontiguousarray(c, dtype=np.int32) for c in (kind, small, graph, dir, nsrc)]
    count = len(cols[0])
    if any(len(c) != count for c in cols):
        raise ValueError("columns differ in length")
    out = np.zeros(max(count, 1), np.int32)
    nu = ctypes.c_int32()
    _check(load().scc_debug_serve_unit(count, *[_ptr(c) for c in cols], int(bool(merge_reach)), batch_graphs,
                                       batch_min, _ptr(out), ctypes.byref(nu)), "scc_debug_serve_unit")
    return out[:nu.value].tolist()


class SccBatch:
    """Owning wrapper of a batch handle: ``SccBatch(packed)`` for a
    :class:`graphgen.Packed` batch (or the four packed arrays)."""

    def __init__(self, packed, stream=None, config: scc_batch_config | None = None):
        self.G = int(packed.G)
        self.nv = int(packed.vbase[-1])
        self.h = scc_batch_create(self.G, packed.vbase, packed.ebase, packed.offsets, packed.targets, stream)
        if config is not None:
            scc_batch_set_config(self.h, config)

    def close(self):
        if getattr(self, "h", None):
            scc_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def labels(self, out=None, stream=None):
        if out is None:
            import torch
            out = torch.empty(max(self.nv, 1), dtype=torch.int32, device="cuda")
        scc_batch_run(self.h, out, stream)
        return out

    def stats(self) -> dict:
        return scc_batch_get_stats(self.h)


# ------------------------------------------------------------------ serving --
def scc_server_config_default() -> scc_server_config:
    c = scc_server_config()
    _check(load().scc_server_config_default(ctypes.byref(c)), "scc_server_config_default")
    return c


class SccServer:
    """A request server (include/scc_serve.h). Host arrays handed to the submit
    calls are kept referenced here until their request has been waited for or
    drained, so the caller may drop them at once."""

    def __init__(self, config: scc_server_config | None = None):
        h = ctypes.c_void_p()
        _check(load().scc_server_create(ctypes.byref(config) if config is not None else None, ctypes.byref(h)),
               "scc_server_create")
        self.h = h.value
        self._keep = {}
        self._graph_n = {}  # vertices of each resident graph (reach outputs hold one mask per vertex)

    def add_graph(self, n: int, offsets, targets) -> int:
        gid = ctypes.c_int32()
        what = "scc_server_add_graph"
        m = _elements(targets)
        po = _arr(offsets, what + " offsets", I32, max(n, 0) + 1)
        _check(load().scc_server_add_graph(self.h, n, m, po, _arr(targets, what + " targets", I32, m),
                                           ctypes.byref(gid)), what)
        self._graph_n[gid.value] = n
        return gid.value

    def remove_graph(self, gid: int) -> None:
        _check(load().scc_server_remove_graph(self.h, gid), "scc_server_remove_graph")
        self._graph_n.pop(gid, None)

    def submit_scc(self, n: int, offsets, targets, labels_out) -> int:
        rid = ctypes.c_int64()
        what = "scc_server_submit_scc"
        m = _elements(targets)
        po = _arr(offsets, what + " offsets", I32, max(n, 0) + 1)
        pt = _arr(targets, what + " targets", I32, m)
        pl = _arr(labels_out, what + " labels_out", I32, max(n, 0))
        _check(load().scc_server_submit_scc(self.h, n, m, po, pt, pl, ctypes.byref(rid)), what)
        self._keep[rid.value] = (offsets, targets, labels_out)
        return rid.value

    def submit_reach(self, gid: int, sources, dir: int, out) -> int:
        rid = ctypes.c_int64()
        src = np.ascontiguousarray(sources, dtype=np.int32)
        _check(load().scc_server_submit_reach(self.h, gid, _ptr(src), len(src), dir,
                                              _arr(out, "scc_server_submit_reach out", W64, self._graph_n.get(gid, 0)),
                                              ctypes.byref(rid)),
               "scc_server_submit_reach")
        self._keep[rid.value] = (out,)
        return rid.value

    def wait(self, rid: int):
        """(status, latency_ms) of a request, after it completed."""
        st, lat = ctypes.c_int32(), ctypes.c_double()
        _check(load().scc_server_wait(self.h, rid, ctypes.byref(st), ctypes.byref(lat)), "scc_server_wait")
        self._keep.pop(rid, None)
        return st.value, lat.value

    def drain(self) -> None:
        _check(load().scc_server_drain(self.h), "scc_server_drain")
        self._keep.clear()

    def stats(self) -> dict:
        s = scc_server_stats()
        _check(load().scc_server_get_stats(self.h, ctypes.byref(s)), "scc_server_get_stats")
        return s.as_dict()

    def reset_stats(self) -> None:
        _check(load().scc_server_reset_stats(self.h), "scc_server_reset_stats")

    def close(self):
        if getattr(self, "h", None):
            _check(load().scc_server_destroy(self.h), "scc_server_destroy")
            self.h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# -------------------------------------------------------------- debug hooks --
def scc_graph_info(h):
    n, m, mt = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().scc_graph_info(h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(mt)), "scc_graph_info")
    return n.value, m.value, mt.value


def scc_debug_csr(h, which: int, off, adj, stream=None) -> None:
    _check(load().scc_debug_csr(h, which, _ptr(off), _ptr(adj), _stream(stream)), "scc_debug_csr")


def scc_debug_trim(h, flags, stream=None) -> None:
    _check(load().scc_debug_trim(h, _ptr(flags), _stream(stream)), "scc_debug_trim")


def scc_debug_pivot_order(h, order, stream=None) -> int:
    na = ctypes.c_int32()
    _check(load().scc_debug_pivot_order(h, _ptr(order), ctypes.byref(na), _stream(stream)), "scc_debug_pivot_order")
    return na.value


def scc_debug_single_reach(h, labels, s: int, dir: int, visited, stream=None) -> None:
    _check(load().scc_debug_single_reach(h, _ptr(labels), s, dir, _ptr(visited), _stream(stream)),
           "scc_debug_single_reach")


def scc_debug_multi_reach(h, labels, sources, k: int, dir: int, pairs, cap: int, table_cap: int = 0,
                          stream=None) -> int:
    npairs = ctypes.c_int64()
    _check(load().scc_debug_multi_reach(h, _ptr(labels), _ptr(sources), k, dir, _ptr(pairs), cap,
                                        ctypes.byref(npairs), table_cap, _stream(stream)), "scc_debug_multi_reach")
    return npairs.value


def scc_debug_reach_multi_wide(h, sources, k: int, dir: int, out, stream=None) -> None:
    _check(load().scc_debug_reach_multi_wide(h, _ptr(sources), k, dir, _ptr(out), _stream(stream)),
           "scc_debug_reach_multi_wide")


def scc_debug_hashbag(items, count: int, lam: int, sigma: int, out, stream=None):
    nout, chunks = ctypes.c_int64(), ctypes.c_int32()
    _check(load().scc_debug_hashbag(_ptr(items), count, lam, sigma, _ptr(out), ctypes.byref(nout),
                                    ctypes.byref(chunks), _stream(stream)), "scc_debug_hashbag")
    return nout.value, chunks.value


def scc_debug_pair_table(keys, count: int, init_cap: int, out, stream=None):
    nout, res = ctypes.c_int64(), ctypes.c_int32()
    _check(load().scc_debug_pair_table(_ptr(keys), count, init_cap, _ptr(out), ctypes.byref(nout),
                                       ctypes.byref(res), _stream(stream)), "scc_debug_pair_table")
    return nout.value, res.value


def scc_debug_launch_count() -> int:
    return int(load().scc_debug_launch_count())


def scc_debug_barrier_timeout(absent_block: int, limit_ns: int, stream=None) -> tuple[int, int]:
    """(return code, blocks that passed) of one grid barrier with a limited wait
    where block ``absent_block`` (-1: none) never arrives; the code is returned,
    not raised, since SCC_ERR_TIMEOUT is the expected outcome of a test."""
    arrived = ctypes.c_int32()
    rc = load().scc_debug_barrier_timeout(absent_block, limit_ns, ctypes.byref(arrived), _stream(stream))
    return int(rc), arrived.value


# ------------------------------------------------------------- convenience --
class SccGraph:
    """Owning wrapper of a graph handle: ``SccGraph(n, offsets, targets)``."""

    def __init__(self, n: int, offsets, targets, stream=None, config: scc_config | None = None):
        self.n = int(n)
        self.m = int(len(targets))
        self.h = scc_graph_create(self.n, self.m, offsets, targets, stream)
        if config is not None:
            scc_set_config(self.h, config)

    def close(self):
        if getattr(self, "h", None):
            scc_graph_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def labels(self, out=None, stream=None):
        """SCC labels (min vertex id per SCC) into ``out`` (device tensor or host array)."""
        if out is None:
            import torch
            out = torch.empty(self.n, dtype=torch.int32, device="cuda")
        scc_run(self.h, out, stream)
        return out

    def reach(self, sources, dir: int = 0, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.n, dtype=torch.int64, device="cuda")
        reach_multi(self.h, sources, len(sources), dir, out, stream)
        return out

    def stats(self) -> dict:
        return scc_get_stats(self.h)
