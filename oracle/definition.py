"""The definitions written out through the transitive closure (numpy) -- test
infrastructure only, for graphs small enough for an n-by-n boolean matrix.

These pin the C oracle: they share none of its code and compute each quantity
straight from its definition.

* ``closure(n, edges)[u, v]`` is True iff u ~> v (a path, possibly empty, from u
  to v; Sec. 1 notation).
* SCC label (Sec. 1 problem statement, canonical minimum):
  ``label[v] = min{u : u ~> v and v ~> u}``.
* Connected component label (Sec. 5.1, connectivity on the symmetrised graph):
  ``label[v] = min{u : u and v joined by a path of arcs taken in either
  direction}``.
* Least-element list (Sec. 5.2, unweighted, undirected graph under the arcs):
  source ``order[j]`` is in L(v) iff ``d(v, order[j]) < min_{k<j} d(v, order[k])``.
* Forward reachability pairs (Sec. 2): ``{(v, s) : s in S, s ~> v}``; backward:
  the same on the transpose. Inside a label class (Alg. 1, MultiReach skips an
  arc (u, v) with L(u) != L(v)) the closure is taken over the subgraph whose arcs
  join two vertices of one class.
"""
from __future__ import annotations

import numpy as np


def adjacency(n: int, edges) -> np.ndarray:
    a = np.zeros((n, n), dtype=bool)
    for u, v in edges:
        a[u, v] = True
    return a


def closure_of(a: np.ndarray) -> np.ndarray:
    """Reflexive-transitive closure by repeated squaring of (I | A)."""
    n = a.shape[0]
    r = a | np.eye(n, dtype=bool)
    while True:
        r2 = (r.astype(np.int64) @ r.astype(np.int64)) > 0
        if np.array_equal(r2, r):
            return r
        r = r2


def closure(n: int, edges) -> np.ndarray:
    return closure_of(adjacency(n, edges))


def scc_labels(n: int, edges) -> np.ndarray:
    """label[v] = min{u : u ~> v and v ~> u}."""
    r = closure(n, edges)
    mutual = r & r.T
    lab = np.empty(n, np.int32)
    for v in range(n):
        lab[v] = int(np.flatnonzero(mutual[:, v])[0])
    return lab


def class_closure(n: int, edges, labels) -> np.ndarray:
    """Closure of the subgraph that keeps arcs (u, v) with labels[u] == labels[v]
    and both labels >= 0 (vertices with a negative label are finished)."""
    labels = np.asarray(labels)
    kept = [(u, v) for u, v in edges if labels[u] == labels[v] and labels[u] >= 0]
    r = closure(n, kept)
    fin = labels < 0
    r[fin, :] = False
    r[:, fin] = False
    return r


def multi_reach_pairs(n: int, edges, labels, sources, backward: bool = False) -> np.ndarray:
    """Sorted uint64 ``v << 32 | s`` for every source s and v with s ~> v (forward)
    or v ~> s (backward) inside s's class."""
    r = class_closure(n, edges, labels)
    if backward:
        r = r.T
    out = set()
    for s in sources:
        for v in np.flatnonzero(r[s]):
            out.add((int(v) << 32) | int(s))
    return np.array(sorted(out), dtype=np.uint64)


def reach_mask(n: int, edges, sources, backward: bool = False) -> np.ndarray:
    """uint64[n] with bit j set iff sources[j] ~> v (forward) or v ~> sources[j]."""
    r = closure(n, edges)
    if backward:
        r = r.T
    out = np.zeros(n, np.uint64)
    for j, s in enumerate(sources):
        out[r[s]] |= np.uint64(1) << np.uint64(j)
    return out


def cc_labels(n: int, edges) -> np.ndarray:
    """label[v] = min{u : u and v are joined by a path of arcs, each taken in
    either direction} (closure of A | A^T)."""
    a = adjacency(n, edges)
    r = closure_of(a | a.T)
    lab = np.empty(n, np.int32)
    for v in range(n):
        lab[v] = int(np.flatnonzero(r[:, v])[0])
    return lab


def bfs_distances(n: int, edges) -> np.ndarray:
    """All-pairs hop distances of the undirected graph under the arcs (-1: unreachable)."""
    a = adjacency(n, edges)
    a = a | a.T
    dist = np.full((n, n), -1, np.int64)
    for s in range(n):
        dist[s, s] = 0
        frontier, d = [s], 0
        while frontier:
            d += 1
            nxt = []
            for u in frontier:
                for w in np.flatnonzero(a[u]):
                    if dist[s, w] < 0:
                        dist[s, w] = d
                        nxt.append(int(w))
            frontier = nxt
    return dist


def le_lists(n: int, edges, order):
    """[[(source, distance), ...] for each v]: order[j] with d(v, order[j])
    smaller than every earlier source's distance, in source order."""
    dist = bfs_distances(n, edges)
    out = []
    for v in range(n):
        best, lst = None, []
        for s in order:
            d = dist[v, s]
            if d >= 0 and (best is None or d < best):
                lst.append((int(s), int(d)))
                best = d
        out.append(lst)
    return out
