"""GPU least-element lists (le_lists_run: Alg. 5 with a packed level frontier
and a hash table of visited pairs, Sec. 5.2) are identical to the oracle's
sequential pruned BFS for the same vertex order: the same offsets, sources and
distances, on edge cases, paths, complete graphs, lattices, R-MAT and k-NN
graphs, for host and device buffers, and when the visited-pair table and the
candidate log start small and must grow."""
import numpy as np
import pytest

import oracle
from paper_2303_04934_gb300 import graphgen as gg
from paper_2303_04934_gb300 import scc

from gpu_util import ensure_lib, make_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _get(G, total, host):
    import torch
    n = G.n
    if host:
        order = np.empty(n, np.int32)
        off = np.empty(n + 1, np.int64)
        src = np.empty(max(total, 1), np.int32)
        dist = np.empty(max(total, 1), np.int32)
        scc.le_lists_get(G.h, order, off, src, dist, total)
        return order, off, src[:total], dist[:total]
    order = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    src = torch.empty(max(total, 1), dtype=torch.int32, device="cuda")
    dist = torch.empty(max(total, 1), dtype=torch.int32, device="cuda")
    scc.le_lists_get(G.h, order[:n] if n else order, off, src[:total] if total else src,
                     dist[:total] if total else dist, total)
    torch.cuda.synchronize()
    return order.cpu().numpy()[:n], off.cpu().numpy(), src.cpu().numpy()[:total], dist.cpu().numpy()[:total]


def _check(g, host=False, small=False):
    with make_graph(g, on_device=not host) as G:
        total = scc.scc_debug_le_lists(G.h, 1024, 64) if small else scc.le_lists_run(G.h)
        order, off, src, dist = _get(G, total, host)
        st = scc.le_get_stats(G.h)
    assert sorted(order.tolist()) == list(range(g.n)), g.name
    w_off, w_src, w_dist = oracle.le_lists(g.n, g.offsets, g.targets, order)
    assert np.array_equal(off, w_off), g.name
    assert np.array_equal(src, w_src), g.name
    assert np.array_equal(dist, w_dist), g.name
    assert st["entries"] == total
    return st


def test_edge_cases():
    _check(gg.from_edges(0, [], name="empty"))
    _check(gg.from_edges(1, [], name="one"))
    _check(gg.from_edges(3, [(1, 1)], name="self_loop"))
    _check(gg.from_edges(6, [], name="no_arcs"))
    _check(gg.from_edges(8, [(i, i + 1) for i in range(7)], name="path8"))
    _check(gg.from_edges(5, [(4, 3), (3, 2), (0, 2), (2, 0)], name="mixed"))


def test_small_random_graphs():
    rng = np.random.default_rng(0x1E5)
    for i in range(40):
        n = int(rng.integers(2, 300))
        p = float(rng.choice([0.003, 0.01, 0.05, 0.2]))
        _check(gg.gnp(n, p, seed=700 + i, allow_self=bool(i % 2)))


@pytest.mark.parametrize("make", [
    lambda: gg.from_edges(500, [(i, i + 1) for i in range(499)], name="path500"),
    lambda: gg.from_edges(60, [(i, j) for i in range(60) for j in range(i + 1, 60)], name="complete60"),
    lambda: gg.torus(2, 100, 0.5, seed=51),
    lambda: gg.torus(3, 20, 0.3, seed=52),
    lambda: gg.rmat(14, 8, seed=53),
    lambda: gg.knn(30_000, 3, seed=54),
], ids=["path500", "complete60", "torus2d_100", "torus3d_20", "rmat14", "knn30k"])
def test_graphs_device_and_host(make):
    g = make()
    _check(g, host=False)
    _check(g, host=True)


def test_growth_of_the_table_and_the_log():
    """Starting from 1024 table slots and a 64-entry log, both must grow; the
    lists are still the oracle's."""
    for g in (gg.torus(2, 80, 0.7, seed=61), gg.rmat(13, 8, seed=62)):
        st = _check(g, small=True)
        assert st["launches"] > 1
