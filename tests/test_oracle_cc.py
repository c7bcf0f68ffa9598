"""Pins of the oracle's connected components (Sec. 5.1: connectivity on the
symmetrised graph, the output of Alg. 4) against the definition (closure of
A | A^T), brute force over every small digraph, closed forms and the relation
to strong connectivity. CPU only."""
import numpy as np
import pytest

import oracle
from oracle import definition
from paper_2303_04934_gb300 import graphgen as gg


def _csr(n, edges):
    g = gg.from_edges(n, edges)
    return g.offsets, g.targets


def _all_digraphs(n):
    pairs = [(u, v) for u in range(n) for v in range(n)]
    for mask in range(1 << len(pairs)):
        yield [pairs[i] for i in range(len(pairs)) if mask >> i & 1]


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_cc_exhaustive_small(n):
    """Every digraph with n <= 4, self-loops included (65,536 at n = 4)."""
    for edges in _all_digraphs(n):
        lab, c = oracle.cc_labels(n, *_csr(n, edges))
        want = definition.cc_labels(n, edges)
        assert np.array_equal(lab, want), edges
        assert c == len(np.unique(want))


def test_cc_random_vs_closure():
    rng = np.random.default_rng(0xCC)
    for trial in range(3000):
        n = int(rng.integers(1, 65))
        p = float(rng.choice([0.01, 0.02, 0.05, 0.1, 0.3]))
        g = gg.gnp(n, p, seed=trial + 7, allow_self=bool(trial % 2))
        edges = gg.edges_of(g).tolist()
        lab, _ = oracle.cc_labels(n, g.offsets, g.targets)
        assert np.array_equal(lab, definition.cc_labels(n, edges)), (trial, n, p)


def test_cc_closed_forms():
    # a directed path is one (weak) component, whichever way its arcs point
    n = 700
    for e in ([(i, i + 1) for i in range(n - 1)], [(i + 1, i) for i in range(n - 1)]):
        lab, c = oracle.cc_labels(n, *_csr(n, e))
        assert c == 1 and not lab.any()
    # isolated vertices and self-loops only: label[v] = v
    lab, c = oracle.cc_labels(5, *_csr(5, [(1, 1), (3, 3)]))
    assert c == 5 and lab.tolist() == [0, 1, 2, 3, 4]
    # disjoint cycles under shuffled ids: one label per cycle, its smallest id
    rng = np.random.default_rng(3)
    sizes = [1, 2, 3, 7, 40]
    perm = rng.permutation(sum(sizes))
    edges, want, s0 = [], np.empty(sum(sizes), np.int32), 0
    for k in sizes:
        ids = perm[s0:s0 + k]
        edges += [(int(ids[i]), int(ids[(i + 1) % k])) for i in range(k)]
        want[ids] = ids.min()
        s0 += k
    lab, c = oracle.cc_labels(len(perm), *_csr(len(perm), edges))
    assert c == len(sizes) and np.array_equal(lab, want)
    # two components joined by one arc, in either direction, become one
    e = [(0, 1), (1, 2), (3, 4), (4, 5)]
    for extra in ((2, 3), (5, 0)):
        lab, c = oracle.cc_labels(6, *_csr(6, e + [extra]))
        assert c == 1 and not lab.any()
    # a torus with every arc present is connected; with no arcs every vertex is alone
    g = gg.torus(2, 30, 1.0, seed=1)
    assert oracle.cc_labels(g.n, g.offsets, g.targets)[1] == 1
    g = gg.torus(3, 8, 0.0, seed=1)
    lab, c = oracle.cc_labels(g.n, g.offsets, g.targets)
    assert c == g.n and np.array_equal(lab, np.arange(g.n))


def test_cc_refined_by_scc_and_invariants():
    """Every SCC lies inside one component; every arc joins two vertices of one
    component; label[label[v]] = label[v] <= v."""
    for i, g in enumerate([gg.rmat(12, 4, seed=5), gg.torus(2, 50, 0.3, seed=6), gg.knn(3000, 3, seed=7),
                           gg.gnp(500, 0.002, seed=8)]):
        cc, _ = oracle.cc_labels(g.n, g.offsets, g.targets)
        scc, _ = oracle.scc_labels(g.n, g.offsets, g.targets)
        assert np.array_equal(cc[scc], cc), i
        src = np.repeat(np.arange(g.n), np.diff(g.offsets))
        assert np.array_equal(cc[src], cc[g.targets]), i
        assert np.array_equal(cc[cc], cc) and (cc <= np.arange(g.n)).all(), i


def test_cc_pins_catch_following_arcs_one_way():
    """A plausible mistake -- following arcs only forwards (reachability from the
    smallest vertex instead of connectivity) -- disagrees with the definition on
    a small graph the exhaustive pin covers."""
    n, edges = 3, [(1, 0), (1, 2)]
    r = definition.closure(n, edges)  # directed reachability only
    wrong = np.array([int(np.flatnonzero(r[:, v])[0]) for v in range(n)], np.int32)
    assert not np.array_equal(wrong, definition.cc_labels(n, edges))
    assert np.array_equal(oracle.cc_labels(n, *_csr(n, edges))[0], definition.cc_labels(n, edges))
