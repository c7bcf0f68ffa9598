"""GPU scc_run labels are bit-identical to the CPU oracle (iterative Tarjan,
canonical minimum) on small, edge-case and medium graphs, for every
configuration (tau, seeds, beta, lambda, pivot seed) and for host or device
buffers. The labels are canonical, so any scheduling order and configuration
must give the same bytes."""
import itertools

import numpy as np
import pytest

import oracle
from oracle.invariants import check_scc_labels
from paper_2303_04934_gb300 import graphgen as gg
from paper_2303_04934_gb300 import scc

from gpu_util import config, ensure_lib, labels_of, make_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _check(g, cfg=None, host=False):
    want, _ = oracle.scc_labels(g.n, g.offsets, g.targets)
    with make_graph(g, cfg, on_device=not host) as G:
        got = labels_of(G, host=host)
        stats = G.stats()
    assert np.array_equal(got, want), g.name
    return stats


def test_edge_cases():
    _check(gg.from_edges(0, [], name="empty"))
    _check(gg.from_edges(1, [], name="one"))
    _check(gg.from_edges(1, [(0, 0)], name="one_self_loop"))
    _check(gg.from_edges(5, [], name="no_arcs"))
    _check(gg.from_edges(4, [(i, i) for i in range(4)], name="self_loops_only"))
    _check(gg.from_edges(6, [(i, (i + 1) % 6) for i in range(6)], name="cycle"))
    _check(gg.from_edges(6, [(i, i + 1) for i in range(5)], name="chain"))
    _check(gg.from_edges(7, [(i, j) for i in range(7) for j in range(7) if i != j], name="complete"))
    _check(gg.from_edges(6, [(0, 1), (1, 2), (2, 0), (3, 4), (4, 5), (5, 3), (2, 3)], name="two_cycles"))
    _check(gg.from_edges(4, [(0, 1), (0, 1), (1, 0), (1, 0), (2, 3)], name="duplicates"))


def test_all_digraphs_with_three_vertices_and_loops():
    pairs = [(u, v) for u in range(3) for v in range(3)]
    for mask in range(1 << 9):
        e = [pairs[i] for i in range(9) if mask >> i & 1]
        _check(gg.from_edges(3, e, name=f"n3_{mask}"))


def test_random_digraphs():
    for trial in range(120):
        n = 1 + trial % 90
        g = gg.gnp(n, [0.01, 0.03, 0.08, 0.2][trial % 4], seed=1000 + trial, allow_self=trial % 5 == 0)
        _check(g)


@pytest.mark.parametrize("make", [
    lambda: gg.torus(2, 256, 0.5, seed=0x5CC00),          # the 2D 256^2 lattice, p = 0.5
    lambda: gg.torus(2, 100, 0.75, seed=1),
    lambda: gg.torus(3, 32, 0.3, seed=2),
    lambda: gg.torus(3, 24, 0.6, seed=3),
    lambda: gg.paper_lattice(200, 150, 0, seed=4),
    lambda: gg.paper_lattice(200, 150, 1, seed=5),
    lambda: gg.rmat(16, 16, seed=6),
    lambda: gg.rmat(15, 4, seed=7),
    lambda: gg.knn(100000, 5, seed=8),
    lambda: gg.knn(30000, 2, seed=9),
], ids=["torus2d_256", "torus2d_100_p75", "torus3d_32", "torus3d_24_p6", "REC_model", "RECp_model",
        "rmat16", "rmat15_ef4", "knn100k", "knn30k_k2"])
def test_medium_graphs(make):
    g = make()
    st = _check(g)
    assert st["batches"] >= 1


@pytest.mark.parametrize("kw", [dict(tau=1), dict(tau=16, seeds=1), dict(tau=4096), dict(beta=2.0),
                                dict(beta=1.1), dict(lam=1024, sigma=8), dict(seed=12345), dict(seeds=4),
                                dict(dense=0), dict(dense=3), dict(dense=200), dict(sigma=0),
                                dict(sigma=0, lam=1024, tau=16)])
def test_configuration_does_not_change_labels(kw):
    # the R-MAT graph with edge factor 16 takes the dense path (average degree >= 8)
    for g in (gg.torus(2, 64, 0.5, seed=31), gg.rmat(13, 8, seed=32), gg.knn(20000, 5, seed=33),
              gg.rmat(13, 16, seed=34)):
        _check(g, config(**kw))


def test_host_buffers_and_repeat_runs():
    g = gg.torus(3, 20, 0.4, seed=41)
    want, _ = oracle.scc_labels(g.n, g.offsets, g.targets)
    with make_graph(g, on_device=False) as G:
        for _ in range(3):
            assert np.array_equal(labels_of(G, host=True), want)
            assert np.array_equal(labels_of(G, host=False), want)


def test_page_locked_host_input():
    """Page-locked host targets are read by the intake pass directly: aligned
    and unaligned starts, self-loops (the CSR is rebuilt) and a bad target."""
    import torch
    # R-MAT 2^18 (4 M arcs) is read in several chunks, each partitioned while
    # the next one is read; the others in one
    for g in (gg.rmat(14, 8, seed=42), gg.torus(2, 90, 0.5, seed=43),
              gg.gnp(300, 0.02, seed=44, allow_self=True), gg.rmat(18, 16, seed=46)):
        want, _ = oracle.scc_labels(g.n, g.offsets, g.targets)
        for shift in (0, 1, 3):
            buf = torch.zeros(g.m + shift + 1, dtype=torch.int32).pin_memory()
            buf[shift:shift + g.m] = torch.from_numpy(g.targets)
            off = torch.from_numpy(g.offsets).pin_memory()
            with scc.SccGraph(g.n, off, buf[shift:shift + g.m]) as G:
                assert np.array_equal(labels_of(G, host=True), want), (g.name, shift)
    g = gg.torus(2, 20, 0.5, seed=45)
    bad = torch.from_numpy(g.targets.copy()).pin_memory()
    bad[len(bad) // 2] = g.n
    with pytest.raises(scc.SccError):
        scc.SccGraph(g.n, torch.from_numpy(g.offsets).pin_memory(), bad)


def _with_self_loops(g, count, seed):
    """g with a self-loop added at the start of `count` random rows."""
    rng = np.random.default_rng(seed)
    sel = np.zeros(g.n, bool)
    sel[rng.choice(g.n, count, replace=False)] = True
    deg = np.diff(g.offsets.astype(np.int64))
    off = np.zeros(g.n + 1, np.int64)
    off[1:] = np.cumsum(deg + sel)
    adj = np.empty(int(off[-1]), np.int32)
    adj[off[:-1][sel]] = np.flatnonzero(sel)
    rows = np.repeat(np.arange(g.n), deg)
    within = np.arange(g.m) - np.repeat(g.offsets[:-1].astype(np.int64), deg)
    adj[(off[:-1] + sel)[rows] + within] = g.targets
    return gg.Graph(g.n, off.astype(np.int32), adj, g.name + "_self")


def test_page_locked_host_input_in_chunks_with_self_loops_and_a_bad_target():
    """A host graph large enough to be read in several chunks, with self-loops:
    the forward CSR is rebuilt without them after the chunked intake and G^T is
    built again in one chunk; a bad target in a late chunk is refused."""
    import torch
    g = _with_self_loops(gg.rmat(18, 16, seed=47), 5000, seed=48)
    assert g.m > 3_500_000  # 7 chunks of whole 8,192-arc tiles
    want, _ = oracle.scc_labels(g.n, g.offsets, g.targets)
    off = torch.from_numpy(g.offsets).pin_memory()
    adj = torch.from_numpy(g.targets).pin_memory()
    with scc.SccGraph(g.n, off, adj) as G:
        n, m, mt = scc.scc_graph_info(G.h)
        assert (n, m, mt) == (g.n, g.m, g.m - 5000)
        assert np.array_equal(labels_of(G, host=True), want)
    bad = adj.clone().pin_memory()
    bad[int(0.8 * g.m)] = g.n
    with pytest.raises(scc.SccError):
        scc.SccGraph(g.n, off, bad)


@pytest.mark.parametrize("make", [
    lambda: gg.rmat(14, 8, seed=61),
    lambda: gg.rmat(13, 16, seed=62),                     # dense rounds (average degree >= 8)
    lambda: gg.torus(2, 64, 0.5, seed=63),
    lambda: gg.knn(20000, 5, seed=64),
    lambda: gg.gnp(400, 0.004, seed=65, allow_self=True),
    lambda: gg.from_edges(50, [(i, i + 1) for i in range(49)], name="chain"),  # one trim pass: the two ends
], ids=["rmat14", "rmat13_ef16", "torus2d_64", "knn20k", "gnp_sparse_self", "chain"])
def test_trim_and_first_scc_counts_match_the_oracle(make):
    """The trimmed vertices (Sec. 4.1) and the size of the first pivot's SCC
    (Sec. 4.2; the pivot is the first of the seeded order over the untrimmed
    vertices) equal the oracle's."""
    g = make()
    want, _ = oracle.scc_labels(g.n, g.offsets, g.targets)
    trimmed = oracle.trim(g.n, g.offsets, g.targets).astype(bool)
    with make_graph(g) as G:
        assert np.array_equal(labels_of(G), want)
        st = G.stats()
    assert st["n_trimmed"] == int(trimmed.sum())
    order = oracle.pivot_order((~trimmed).astype(np.uint8), seed=scc.scc_config_default().seed)
    first = int((want == want[order[0]]).sum()) if len(order) else 0
    assert st["first_scc_size"] == first


def test_invariants_hold_on_gpu_output():
    g = gg.rmat(15, 8, seed=51)
    with make_graph(g) as G:
        lab = labels_of(G)
    check_scc_labels(g.n, g.offsets, g.targets, lab)


def _shuffled(n, edges, seed, name):
    """The same graph with vertex ids permuted (so structure and ids do not align)."""
    p = np.random.default_rng(seed).permutation(n)
    return gg.from_edges(n, [(int(p[a]), int(p[b])) for a, b in edges], name=name)


def test_deep_and_skewed_structures():
    """Long chains and cycles (searches thousands of levels deep, so many rounds),
    a hub with 200k out- and in-arcs (hub items cut into segments), cycles tied
    into a DAG by chains, and a complete bipartite orientation (one huge level)."""
    n = 30000
    _check(_shuffled(n, [(i, i + 1) for i in range(n - 1)], 1, "path30k"))
    _check(_shuffled(n, [(i, (i + 1) % n) for i in range(n)], 2, "cycle30k"))
    # two long cycles joined one way, plus a tail
    e = [(i, (i + 1) % 10000) for i in range(10000)] + [(10000 + i, 10000 + (i + 1) % 10000) for i in range(10000)]
    e += [(5, 10005)] + [(20000 + i, 20001 + i) for i in range(4999)] + [(10007, 20000)]
    _check(_shuffled(25000, e, 3, "cycles_and_tail"))
    # a star: hub 0 -> every leaf, every leaf -> hub (one SCC), plus leaves with one direction only
    k = 200000
    e = [(0, i) for i in range(1, k)] + [(i, 0) for i in range(1, k, 2)]
    _check(gg.from_edges(k, e, name="star200k"))
    # complete bipartite orientation: every arc from side A to side B, a few back arcs
    a, b = 300, 300
    e = [(i, a + j) for i in range(a) for j in range(b)] + [(a + j, j) for j in range(0, a, 7)]
    _check(_shuffled(a + b, e, 4, "bipartite"))
    # a deep ring of small cliques (many small SCCs along a long chain)
    e = []
    for c in range(3000):
        base = 4 * c
        e += [(base + x, base + y) for x in range(4) for y in range(4) if x != y]
        e.append((base + 3, base + 4)) if c < 2999 else None
    _check(_shuffled(12000, e, 5, "clique_chain"))
