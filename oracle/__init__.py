"""CPU oracle for the SCC hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference leg may import this package. It shares no code with the CUDA path
(``paper_2303_04934_gb300``) and never imports it.

* :mod:`oracle.scc_oracle` (``scc_oracle.c``, plain C): iterative Tarjan, the
  transpose, trimming, class-restricted single/multi reachability, plain
  multi-source reachability masks, the seeded pivot order and batch bounds,
  connected components of the undirected graph under the arcs (Sec. 5.1) and
  its least-element lists for a vertex order (Sec. 5.2).
* :mod:`oracle.definition` (numpy): the definitions written out through the
  transitive closure, for tiny graphs -- the pins of the C oracle.
* :mod:`oracle.invariants` (numpy): properties every correct SCC labelling has.
* :mod:`oracle.bgss_model` (plain Python): the method's own steps (Alg. 1) with
  the library's readings, sequentially on small graphs; its labels must be
  Tarjan's.

Paper: Wang, Dong, Gu, Sun, "Parallel Strong Connectivity Based on Faster
Reachability" (SIGMOD 2023); section and algorithm numbers in the docstrings
refer to it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scc_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_lib")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile scc_oracle.c into ``oracle/_lib/liboracle.so`` with gcc."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-std=gnu11", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            vp, i64, i32, u64, dbl = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                      ctypes.c_uint64, ctypes.c_double)
            lib.or_scc_tarjan.argtypes = [i64, vp, vp, vp]
            lib.or_transpose.argtypes = [i64, vp, vp, vp, vp]
            lib.or_trim.argtypes = [i64, vp, vp, vp]
            lib.or_reach_set.argtypes = [i64, vp, vp, vp, i32, vp]
            lib.or_multi_reach.argtypes = [i64, vp, vp, vp, vp, i64, vp, i64]
            lib.or_reach_mask.argtypes = [i64, vp, vp, vp, i64, vp]
            lib.or_pivot_order.argtypes = [i64, vp, u64, vp]
            lib.or_batch_bounds.argtypes = [i64, dbl, vp, i64]
            lib.or_cc_labels.argtypes = [i64, vp, vp, vp]
            lib.or_le_lists.argtypes = [i64, vp, vp, vp, vp, vp, vp, i64]
            lib.or_mix64.argtypes = [u64]
            lib.or_mix64.restype = u64
            for f in ("or_scc_tarjan", "or_transpose", "or_trim", "or_reach_set", "or_multi_reach",
                      "or_reach_mask", "or_pivot_order", "or_batch_bounds", "or_cc_labels", "or_le_lists"):
                getattr(lib, f).restype = i64
            _lib = lib
    return _lib


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


def _csr(offsets, targets):
    off, po = _c(offsets, np.int32)
    adj, pa = _c(targets if len(targets) else np.zeros(1, np.int32), np.int32)
    return off, po, adj, pa


def scc_labels(n: int, offsets, targets):
    """SCC labels by iterative Tarjan (Sec. 1 problem statement; SEQ of Sec. 6):
    ``label[v]`` = smallest vertex id in v's SCC. Returns (labels int32[n], #SCC)."""
    off, po, adj, pa = _csr(offsets, targets)
    lab = np.empty(max(n, 1), np.int32)
    c = _load().or_scc_tarjan(n, po, pa, lab.ctypes.data)
    if c < 0:
        raise MemoryError("oracle: Tarjan allocation failed")
    return lab[:n], int(c)


def cc_labels(n: int, offsets, targets):
    """Connected components of the undirected graph under the arcs (Sec. 5.1,
    Alg. 4 output; the paper symmetrises directed inputs): ``label[v]`` =
    smallest vertex id of v's component, by a sequential union-find. Returns
    (labels int32[n], #components)."""
    off, po, adj, pa = _csr(offsets, targets)
    lab = np.empty(max(n, 1), np.int32)
    c = _load().or_cc_labels(n, po, pa, lab.ctypes.data)
    if c < 0:
        raise MemoryError("oracle: union-find allocation failed")
    return lab[:n], int(c)


def le_lists(n: int, offsets, targets, order):
    """Least-element lists (Sec. 5.2) of the undirected graph under the arcs for
    the vertex order ``order``: returns (le_off int64[n+1], le_src int32[],
    le_dist int32[]) with L(u) = le_src[le_off[u]:le_off[u+1]] in source order
    (distances strictly decreasing), by the sequential pruned BFS."""
    off, po, adj, pa = _csr(offsets, targets)
    o, pord = _c(order if len(order) else np.zeros(1, np.int32), np.int32)
    le_off = np.zeros(n + 1, np.int64)
    cap = 4 * n + 16
    while True:
        src = np.empty(max(cap, 1), np.int32)
        dst = np.empty(max(cap, 1), np.int32)
        t = _load().or_le_lists(n, po, pa, pord, le_off.ctypes.data, src.ctypes.data, dst.ctypes.data, cap)
        if t < 0:
            raise MemoryError("oracle: LE-lists allocation failed")
        if t <= cap:
            return le_off, src[:t], dst[:t]
        cap = t


def transpose(n: int, offsets, targets):
    """G^T without self-loops; each row lists its in-neighbours in increasing order."""
    off, po, adj, pa = _csr(offsets, targets)
    toff = np.empty(n + 1, np.int32)
    tadj = np.empty(max(len(targets), 1), np.int32)
    mt = _load().or_transpose(n, po, pa, toff.ctypes.data, tadj.ctypes.data)
    return toff, tadj[:mt]


def trim(n: int, offsets, targets):
    """Trim flags (Sec. 4.1): 1 where v has no out-arc or no in-arc (self-loops not counted)."""
    off, po, adj, pa = _csr(offsets, targets)
    fl = np.empty(max(n, 1), np.uint8)
    _load().or_trim(n, po, pa, fl.ctypes.data)
    return fl[:n]


def reach_set(n: int, offsets, targets, s: int, labels=None):
    """uint8[n]: vertices reached from s over arcs that stay inside label[s]'s class
    (labels None = one class). Pass G^T's CSR for a backward search."""
    off, po, adj, pa = _csr(offsets, targets)
    lp = None
    if labels is not None:
        lab, lp = _c(labels, np.int32)
    vis = np.empty(max(n, 1), np.uint8)
    _load().or_reach_set(n, po, pa, lp, int(s), vis.ctypes.data)
    return vis[:n]


def multi_reach(n: int, offsets, targets, labels, sources):
    """Pair set of a class-restricted multi-reachability search (Sec. 2; Alg. 1):
    uint64 array of ``v << 32 | s`` for every source s and every v it reaches
    inside its class, sorted. Pass G^T's CSR for the backward search."""
    off, po, adj, pa = _csr(offsets, targets)
    lab, lp = _c(labels, np.int32)
    src, sp = _c(sources if len(sources) else np.zeros(1, np.int32), np.int32)
    k = len(sources)
    lib = _load()
    total = lib.or_multi_reach(n, po, pa, lp, sp, k, None, 0)
    if total < 0:
        raise MemoryError("oracle: multi_reach allocation failed")
    out = np.empty(max(total, 1), np.uint64)
    lib.or_multi_reach(n, po, pa, lp, sp, k, out.ctypes.data, total)
    return np.sort(out[:total])


def reach_mask(n: int, offsets, targets, sources):
    """uint64[n]: bit j set where sources[j] reaches v (plain reachability, k <= 64)."""
    off, po, adj, pa = _csr(offsets, targets)
    src, sp = _c(sources, np.int32)
    out = np.empty(max(n, 1), np.uint64)
    if _load().or_reach_mask(n, po, pa, sp, len(sources), out.ctypes.data) < 0:
        raise ValueError("oracle: bad sources")
    return out[:n]


def pivot_order(active, seed: int):
    """Seeded pivot order over the active vertices (Alg. 1 random partition into
    batches): a Feistel bijection with cycle walking applied to their increasing list."""
    act, ap = _c(active, np.uint8)
    n = len(act)
    out = np.empty(max(n, 1), np.int32)
    N = _load().or_pivot_order(n, ap, seed & (2**64 - 1), out.ctypes.data)
    return out[:N]


def mix64(z: int) -> int:
    """The SplitMix64 finaliser the pivot order's Feistel rounds use."""
    return int(_load().or_mix64(z & (2**64 - 1)))


def batch_bounds(N: int, beta: float):
    """Prefix-doubling batch bounds (sizes ceil(beta^i), iterated in double)."""
    lib = _load()
    nb = lib.or_batch_bounds(N, beta, None, -1)
    b = np.empty(nb + 1, np.int64)
    lib.or_batch_bounds(N, beta, b.ctypes.data, nb)
    return b
