"""Pins of the oracle's least-element lists (Sec. 5.2, unweighted, on the
undirected graph under the arcs) against the definition (all-pairs BFS
distances and the running minimum over the source order), brute force over
every small digraph and many orders, closed forms and the expected list length.
CPU only."""
import numpy as np
import pytest

import oracle
from oracle import definition
from paper_2303_04934_gb300 import graphgen as gg


def _csr(n, edges):
    g = gg.from_edges(n, edges)
    return g.offsets, g.targets


def _lists(n, le_off, src, dist):
    return [list(zip(src[le_off[v]:le_off[v + 1]].tolist(), dist[le_off[v]:le_off[v + 1]].tolist()))
            for v in range(n)]


def _all_digraphs(n):
    pairs = [(u, v) for u in range(n) for v in range(n) if u < v]  # undirected: one arc per pair suffices
    for mask in range(1 << len(pairs)):
        yield [pairs[i] for i in range(len(pairs)) if mask >> i & 1]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_le_lists_exhaustive_small(n):
    """Every simple graph on n <= 5 vertices under 6 orders each (and arcs taken either way)."""
    rng = np.random.default_rng(n)
    for edges in _all_digraphs(n):
        for t in range(6):
            order = rng.permutation(n).astype(np.int32)
            es = [(v, u) if (t + u) % 2 else (u, v) for u, v in edges]  # arc directions do not matter
            got = _lists(n, *oracle.le_lists(n, *_csr(n, es), order))
            assert got == definition.le_lists(n, es, order), (edges, order)


def test_le_lists_random_vs_definition():
    rng = np.random.default_rng(0x1E)
    for trial in range(600):
        n = int(rng.integers(1, 60))
        p = float(rng.choice([0.02, 0.05, 0.1, 0.3]))
        g = gg.gnp(n, p, seed=trial + 11, allow_self=bool(trial % 3 == 0))
        edges = gg.edges_of(g).tolist()
        order = rng.permutation(n).astype(np.int32)
        got = _lists(n, *oracle.le_lists(n, g.offsets, g.targets, order))
        assert got == definition.le_lists(n, edges, order), (trial, n, p)


def test_le_lists_closed_forms():
    n = 200
    path = [(i, i + 1) for i in range(n - 1)]
    ident = np.arange(n, dtype=np.int32)
    got = _lists(n, *oracle.le_lists(n, *_csr(n, path), ident))
    # identity order on a path: every earlier vertex is closer than the one before it
    assert all(got[v] == [(j, v - j) for j in range(v + 1)] for v in range(n))
    got = _lists(n, *oracle.le_lists(n, *_csr(n, path), ident[::-1].copy()))
    assert all(got[v] == [(j, j - v) for j in range(n - 1, v - 1, -1)] for v in range(n))
    # complete graph: the first source at distance 1, then the vertex itself
    n = 30
    comp = [(i, j) for i in range(n) for j in range(i + 1, n)]
    order = np.random.default_rng(2).permutation(n).astype(np.int32)
    got = _lists(n, *oracle.le_lists(n, *_csr(n, comp), order))
    o0 = int(order[0])
    assert all(got[v] == ([(v, 0)] if v == o0 else [(o0, 1), (v, 0)]) for v in range(n))
    # isolated vertices (self-loops change nothing): only themselves
    got = _lists(4, *oracle.le_lists(4, *_csr(4, [(1, 1)]), np.array([3, 1, 0, 2], np.int32)))
    assert got == [[(0, 0)], [(1, 0)], [(2, 0)], [(3, 0)]]


def test_le_lists_structure_and_expected_length():
    """Lists end with the vertex itself at distance 0, distances strictly
    decrease, and the mean length under a random order is about ln n plus a
    constant (the expected O(log n) of Sec. 5.2)."""
    g = gg.torus(2, 60, 1.0, seed=3)
    order = np.random.default_rng(5).permutation(g.n).astype(np.int32)
    le_off, src, dist = oracle.le_lists(g.n, g.offsets, g.targets, order)
    rank = np.empty(g.n, np.int64)
    rank[order] = np.arange(g.n)
    for v in range(g.n):
        s, d = src[le_off[v]:le_off[v + 1]], dist[le_off[v]:le_off[v + 1]]
        assert s[-1] == v and d[-1] == 0
        assert (np.diff(d) < 0).all() and (np.diff(rank[s]) > 0).all()
    mean = (le_off[-1]) / g.n
    assert 0.5 * np.log(g.n) < mean < 3 * np.log(g.n)


def test_le_lists_pins_catch_non_strict_minimum():
    """A plausible mistake -- keeping a source whose distance only ties the
    running minimum -- disagrees with the definition on a tiny graph."""
    n, edges, order = 3, [(0, 1), (1, 2)], [0, 2, 1]
    dist = definition.bfs_distances(n, edges)
    wrong = []
    for v in range(n):
        best, lst = None, []
        for s in order:
            if best is None or dist[v, s] <= best:
                lst.append((s, int(dist[v, s])))
                best = dist[v, s]
        wrong.append(lst)
    assert wrong != definition.le_lists(n, edges, order)
    assert _lists(n, *oracle.le_lists(n, *_csr(n, edges), np.array(order, np.int32))) == \
        definition.le_lists(n, edges, order)
