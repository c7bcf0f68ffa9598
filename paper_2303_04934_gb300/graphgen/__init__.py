"""Seeded synthetic input graphs (int32 CSR) shared by the tests, the benchmark and
the oracle's tests.

This module produces inputs only; it holds none of the SCC method's arithmetic.
The generators are host C (``graphgen.c``, OpenMP) and every draw is a
counter-based SplitMix64 value, so a graph depends only on its parameters and
seed.  ``build()`` compiles the library with gcc; the first call of any
generator builds it on demand.

Families (the lattice models follow the paper's Sec. 6 "Setup"):

* :func:`torus` - 2D/3D torus, each of the 2*dims neighbour arcs present
  independently with probability ``p``.
* :func:`paper_lattice` - the paper's SQR/REC (model 0) and SQR'/REC' (model 1).
* :func:`rmat` - R-MAT, self-loops and duplicates removed, ids permuted.
* :func:`knn` - directed k-NN graph of a Gaussian mixture in the unit cube.
* :func:`gnp` - small uniform random digraphs for tests.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_OUT_DIR = os.path.join(os.path.dirname(_HERE), "_lib")
_SO = os.path.join(_OUT_DIR, "libgraphgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile graphgen.c into ``_lib/libgraphgen.so`` (gcc, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=gnu11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            i64, i32p, f32p, u64, dbl, cint = (ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_uint64, ctypes.c_double, ctypes.c_int)
            lib.gg_torus.argtypes = [cint, i64, i64, i64, dbl, u64, i32p, i32p, cint]
            lib.gg_torus.restype = i64
            lib.gg_paper_lattice.argtypes = [i64, i64, cint, u64, i32p, i32p, cint]
            lib.gg_paper_lattice.restype = i64
            lib.gg_rmat.argtypes = [cint, i64, dbl, dbl, dbl, u64, cint, i32p, i32p, cint]
            lib.gg_rmat.restype = i64
            lib.gg_knn.argtypes = [i64, cint, dbl, cint, u64, i32p, i32p, f32p, cint]
            lib.gg_knn.restype = i64
            lib.gg_gnp.argtypes = [i64, dbl, cint, u64, i32p, i32p]
            lib.gg_gnp.restype = i64
            _lib = lib
    return _lib


@dataclass
class Graph:
    """A directed graph in int32 CSR form: row v of ``targets`` is
    ``targets[offsets[v]:offsets[v+1]]`` (the out-neighbours of v)."""
    n: int
    offsets: np.ndarray  # int32[n+1]
    targets: np.ndarray  # int32[m]
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.offsets[-1]) if self.n >= 0 and len(self.offsets) else 0


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def _finish(n, off, adj, m, name):
    if m < 0:
        raise ValueError(f"graphgen: bad arguments for {name}")
    return Graph(n, off, adj[:m], name)


def torus(dims: int, side, p: float, seed: int, threads: int = 0) -> Graph:
    """Torus lattice; ``side`` is an int (same on every axis) or a tuple."""
    if isinstance(side, int):
        side = (side,) * dims
    X, Y, Z = (list(side) + [1, 1])[:3]
    n = X * Y * Z
    off = np.empty(n + 1, np.int32)
    adj = np.empty(max(1, 2 * dims * n), np.int32)
    m = _load().gg_torus(dims, X, Y, Z, p, seed & (2**64 - 1), _p(off), _p(adj), threads)
    return _finish(n, off, adj, m, f"torus{dims}d_{'x'.join(map(str, side))}_p{p}")


def paper_lattice(X: int, Y: int, model: int, seed: int, threads: int = 0) -> Graph:
    """The paper's SQR/REC (model 0) or SQR'/REC' (model 1) lattice on an X-by-Y torus."""
    n = X * Y
    off = np.empty(n + 1, np.int32)
    adj = np.empty(max(1, 4 * n), np.int32)
    m = _load().gg_paper_lattice(X, Y, model, seed & (2**64 - 1), _p(off), _p(adj), threads)
    return _finish(n, off, adj, m, f"paper_lattice{model}_{X}x{Y}")


def rmat(scale: int, edge_factor: int, seed: int, a=0.57, b=0.19, c=0.19, permute=True,
         threads: int = 0) -> Graph:
    """R-MAT with ``edge_factor * 2**scale`` samples, self-loops and duplicates removed."""
    n = 1 << scale
    ns = edge_factor * n
    off = np.empty(n + 1, np.int32)
    adj = np.empty(max(1, ns), np.int32)
    m = _load().gg_rmat(scale, ns, a, b, c, seed & (2**64 - 1), int(permute), _p(off), _p(adj), threads)
    return _finish(n, off, adj, m, f"rmat_s{scale}_ef{edge_factor}")


def knn(n: int, k: int, seed: int, clusters: int = 64, sigma: float = 0.02, threads: int = 0,
        return_points: bool = False):
    """Directed k-NN graph of ``n`` points from a mixture of isotropic 3D Gaussians."""
    off = np.empty(n + 1, np.int32)
    adj = np.empty(max(1, k * n), np.int32)
    pts = np.empty((max(1, n), 3), np.float32) if return_points else None
    m = _load().gg_knn(n, clusters, sigma, k, seed & (2**64 - 1), _p(off), _p(adj),
                       _p(pts) if pts is not None else None, threads)
    g = _finish(n, off, adj, m, f"knn_n{n}_k{k}")
    return (g, pts[:n]) if return_points else g


def gnp(n: int, p: float, seed: int, allow_self: bool = False) -> Graph:
    """Small uniform random digraph G(n, p) over ordered pairs."""
    off = np.empty(n + 1, np.int32)
    adj = np.empty(max(1, n * n), np.int32)
    m = _load().gg_gnp(n, p, int(allow_self), seed & (2**64 - 1), _p(off), _p(adj))
    return _finish(n, off, adj, m, f"gnp_{n}_{p}")


def from_edges(n: int, edges, name: str = "edges") -> Graph:
    """CSR from an explicit arc list (kept in the given order within each row)."""
    e = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    order = np.argsort(e[:, 0], kind="stable") if len(e) else np.zeros(0, np.int64)
    e = e[order]
    cnt = np.bincount(e[:, 0], minlength=n) if len(e) else np.zeros(n, np.int64)
    off = np.zeros(n + 1, np.int32)
    off[1:] = np.cumsum(cnt)
    return Graph(n, off, e[:, 1].astype(np.int32), name)


def edges_of(g: Graph) -> np.ndarray:
    """(m, 2) int64 array of the arcs of g, row by row."""
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.offsets.astype(np.int64)))
    return np.stack([src, g.targets.astype(np.int64)], axis=1)


# ------------------------------------------------------------------ batches --
@dataclass
class Packed:
    """Many graphs in one int32 CSR with per-graph int64 bases (the layout of
    ``include/scc_batch.h``): graph g has ``n_g = vbase[g+1] - vbase[g]``
    vertices, its ``n_g + 1`` local offsets at ``offsets[vbase[g] + g:]`` and
    its ``m_g = ebase[g+1] - ebase[g]`` local targets at ``targets[ebase[g]:]``."""
    G: int
    vbase: np.ndarray    # int64[G+1]
    ebase: np.ndarray    # int64[G+1]
    offsets: np.ndarray  # int32[vbase[G] + G]
    targets: np.ndarray  # int32[ebase[G]]
    names: list

    def graph(self, g: int) -> Graph:
        n = int(self.vbase[g + 1] - self.vbase[g])
        o0 = int(self.vbase[g]) + g
        e0, e1 = int(self.ebase[g]), int(self.ebase[g + 1])
        return Graph(n, self.offsets[o0:o0 + n + 1], self.targets[e0:e1], self.names[g])

    def labels_of(self, labels, g: int):
        return labels[int(self.vbase[g]):int(self.vbase[g + 1])]


def pack(graphs) -> Packed:
    """Pack a list of :class:`Graph` into one :class:`Packed` batch."""
    G = len(graphs)
    vbase = np.zeros(G + 1, np.int64)
    ebase = np.zeros(G + 1, np.int64)
    for i, g in enumerate(graphs):
        vbase[i + 1] = vbase[i] + g.n
        ebase[i + 1] = ebase[i] + g.m
    offs = [np.asarray(g.offsets[:g.n + 1], np.int32) for g in graphs]
    tgts = [np.asarray(g.targets[:g.m], np.int32) for g in graphs]
    offsets = np.concatenate(offs) if offs else np.zeros(0, np.int32)
    targets = np.concatenate(tgts) if tgts else np.zeros(0, np.int32)
    return Packed(G, vbase, ebase, offsets, targets, [g.name for g in graphs])


def mixed_batch_spec(G: int, n_lo: int, n_hi: int, seed: int):
    """(kind, size, seed) of each graph of a mixed batch: vertex counts
    log-uniform in [n_lo, n_hi]; even entries are 2D tori of side ceil(sqrt(n))
    with p = 0.5, odd entries R-MAT of scale round(log2 n) with edge factor 8."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), G))
    spec = []
    for i, n in enumerate(ns):
        s = (seed * 1000003 + i) & (2**63 - 1)
        if i % 2 == 0:
            spec.append(("torus", int(np.ceil(np.sqrt(n))), s))
        else:
            spec.append(("rmat", max(1, int(round(np.log2(n)))), s))
    return spec


def make_from_spec(item) -> Graph:
    kind, size, s = item
    if kind == "torus":
        return torus(2, size, 0.5, seed=s, threads=1)
    return rmat(size, 8, seed=s, threads=1)


def mixed_batch(G: int, n_lo: int, n_hi: int, seed: int, workers: int = 0) -> Packed:
    """A packed batch of :func:`mixed_batch_spec` graphs (generated in parallel)."""
    import concurrent.futures as cf
    spec = mixed_batch_spec(G, n_lo, n_hi, seed)
    workers = workers or (os.cpu_count() or 1)
    _load()
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        graphs = list(ex.map(make_from_spec, spec))
    return pack(graphs)
