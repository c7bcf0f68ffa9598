"""Pins of the CPU oracle against the definitions (transitive closure), closed
forms and brute force on tiny inputs. CPU only."""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import definition
from paper_2303_04934_gb300 import graphgen as gg


def _csr(n, edges):
    g = gg.from_edges(n, edges)
    return g.offsets, g.targets


def _all_digraphs(n, self_loops):
    pairs = [(u, v) for u in range(n) for v in range(n) if self_loops or u != v]
    for mask in range(1 << len(pairs)):
        yield [pairs[i] for i in range(len(pairs)) if mask >> i & 1]


# ----------------------------------------------------------------- Tarjan --

@pytest.mark.parametrize("n,self_loops", [(1, True), (2, True), (3, True), (4, True)])
def test_tarjan_exhaustive_small(n, self_loops):
    """Every digraph with n <= 4, self-loops included (65,536 at n = 4): Tarjan == definition."""
    count = 0
    for edges in _all_digraphs(n, self_loops):
        off, adj = _csr(n, edges)
        lab, nscc = oracle.scc_labels(n, off, adj)
        want = definition.scc_labels(n, edges)
        assert np.array_equal(lab, want), edges
        assert nscc == len(np.unique(want))
        count += 1
    assert count == 2 ** (n * n if self_loops else n * (n - 1))


def test_tarjan_random_vs_closure():
    rng = np.random.default_rng(0x5CC)
    for trial in range(10_000):
        n = int(rng.integers(1, 65))
        p = float(rng.choice([0.02, 0.05, 0.1, 0.2, 0.5]))
        g = gg.gnp(n, p, seed=trial, allow_self=bool(trial % 3 == 0))
        edges = gg.edges_of(g).tolist()
        lab, _ = oracle.scc_labels(n, g.offsets, g.targets)
        assert np.array_equal(lab, definition.scc_labels(n, edges)), (trial, n, p)


def test_tarjan_duplicate_arcs_and_empty():
    lab, c = oracle.scc_labels(0, np.zeros(1, np.int32), np.zeros(0, np.int32))
    assert len(lab) == 0 and c == 0
    edges = [(0, 1), (0, 1), (1, 0), (1, 0), (2, 2), (2, 2)]
    off, adj = _csr(3, edges)
    lab, c = oracle.scc_labels(3, off, adj)
    assert lab.tolist() == [0, 0, 2] and c == 2


# ------------------------------------------------------------ closed forms --

def test_closed_forms():
    # directed cycle: one SCC labelled 0
    for n in (1, 2, 5, 1000):
        e = [(i, (i + 1) % n) for i in range(n)]
        lab, c = oracle.scc_labels(n, *_csr(n, e))
        assert c == 1 and not lab.any()
    # directed path and any DAG with arcs i<j only: label[v] = v
    n = 500
    lab, c = oracle.scc_labels(n, *_csr(n, [(i, i + 1) for i in range(n - 1)]))
    assert c == n and np.array_equal(lab, np.arange(n))
    rng = np.random.default_rng(1)
    dag = [(int(i), int(j)) for i, j in rng.integers(0, n, (3000, 2)) if i < j]
    lab, c = oracle.scc_labels(n, *_csr(n, dag))
    assert c == n and np.array_equal(lab, np.arange(n))
    # complete digraph: one SCC
    n = 40
    lab, c = oracle.scc_labels(n, *_csr(n, [(i, j) for i in range(n) for j in range(n) if i != j]))
    assert c == 1 and not lab.any()
    # disjoint union of cycles with shuffled ids: one label per cycle = its minimum
    perm = rng.permutation(300)
    sizes = [1, 2, 3, 7, 50, 237]
    edges, start, want = [], 0, np.empty(300, np.int64)
    for s in sizes:
        ids = perm[start:start + s]
        edges += [(int(ids[i]), int(ids[(i + 1) % s])) for i in range(s)] if s > 1 else []
        want[ids] = ids.min()
        start += s
    lab, c = oracle.scc_labels(300, *_csr(300, edges))
    assert c == len(sizes) and np.array_equal(lab, want)
    # two cycles joined by one arc: 2 SCCs
    e = [(0, 1), (1, 2), (2, 0), (3, 4), (4, 5), (5, 3), (2, 3)]
    lab, c = oracle.scc_labels(6, *_csr(6, e))
    assert c == 2 and lab.tolist() == [0, 0, 0, 3, 3, 3]
    # self-loop-only vertices are singletons
    lab, c = oracle.scc_labels(4, *_csr(4, [(i, i) for i in range(4)]))
    assert c == 4 and np.array_equal(lab, np.arange(4))


@pytest.mark.parametrize("dims,side", [(2, 37), (3, 9)])
def test_torus_all_arcs_and_no_arcs(dims, side):
    g = gg.torus(dims, side, 1.0, seed=3)
    assert g.m == 2 * dims * g.n
    lab, c = oracle.scc_labels(g.n, g.offsets, g.targets)
    assert c == 1 and not lab.any()
    g0 = gg.torus(dims, side, 0.0, seed=3)
    lab, c = oracle.scc_labels(g0.n, g0.offsets, g0.targets)
    assert g0.m == 0 and c == g0.n and np.array_equal(lab, np.arange(g0.n))


# --------------------------------------------------- transpose and trimming --

def test_transpose_and_trim_vs_definition():
    for trial in range(200):
        n = 1 + trial % 40
        g = gg.gnp(n, [0.03, 0.1, 0.3][trial % 3], seed=100 + trial, allow_self=True)
        e = gg.edges_of(g)
        toff, tadj = oracle.transpose(n, g.offsets, g.targets)
        # definition: multiset of reversed non-loop arcs, grouped by the new source
        want = sorted((int(v), int(u)) for u, v in e if u != v)
        got = sorted((v, int(u)) for v in range(n) for u in tadj[toff[v]:toff[v + 1]])
        assert got == want
        a = definition.adjacency(n, e.tolist())
        np.fill_diagonal(a, False)
        want_trim = (a.sum(1) == 0) | (a.sum(0) == 0)
        assert np.array_equal(oracle.trim(n, g.offsets, g.targets).astype(bool), want_trim)


# ------------------------------------------------------------ reachability --

def test_reach_set_multi_reach_and_masks_vs_closure():
    rng = np.random.default_rng(7)
    for trial in range(150):
        n = int(rng.integers(2, 48))
        g = gg.gnp(n, float(rng.choice([0.03, 0.08, 0.2])), seed=500 + trial, allow_self=True)
        e = gg.edges_of(g).tolist()
        toff, tadj = oracle.transpose(n, g.offsets, g.targets)
        # random classes, some vertices finished (negative label)
        labels = rng.integers(-1, 3, n).astype(np.int32)
        k = int(rng.integers(1, min(n, 10) + 1))
        sources = rng.choice(n, k, replace=bool(trial % 4 == 0)).astype(np.int32)
        live = sources[labels[sources] >= 0]
        fw = oracle.multi_reach(n, g.offsets, g.targets, labels, sources)
        bw = oracle.multi_reach(n, toff, tadj, labels, sources)
        assert np.array_equal(fw, definition.multi_reach_pairs(n, e, labels, live))
        assert np.array_equal(bw, definition.multi_reach_pairs(n, e, labels, live, backward=True))
        s = int(sources[0])
        rs = oracle.reach_set(n, g.offsets, g.targets, s, labels)
        cl = definition.class_closure(n, e, labels)
        assert np.array_equal(rs.astype(bool), cl[s])
        ksrc = rng.choice(n, min(n, 64), replace=True).astype(np.int32)
        assert np.array_equal(oracle.reach_mask(n, g.offsets, g.targets, ksrc),
                              definition.reach_mask(n, e, ksrc))
        assert np.array_equal(oracle.reach_mask(n, toff, tadj, ksrc),
                              definition.reach_mask(n, e, ksrc, backward=True))


def test_reach_links_to_scc():
    """v in SCC(s) <=> s ~> v and v ~> s <=> label[v] == label[s]."""
    g = gg.rmat(10, 8, seed=11)
    lab, _ = oracle.scc_labels(g.n, g.offsets, g.targets)
    toff, tadj = oracle.transpose(g.n, g.offsets, g.targets)
    src = np.arange(0, g.n, 17, dtype=np.int32)[:64]
    f = oracle.reach_mask(g.n, g.offsets, g.targets, src)
    b = oracle.reach_mask(g.n, toff, tadj, src)
    both = f & b
    for j, s in enumerate(src):
        inscc = (both >> np.uint64(j)) & np.uint64(1)
        assert np.array_equal(inscc.astype(bool), lab == lab[s])


# --------------------------------------------------------- pivots and batches --

def test_batch_bounds_closed_forms():
    # beta = 2: sizes 2^i exactly, bounds 2^i - 1
    b = oracle.batch_bounds(1000, 2.0)
    assert b.tolist() == [0, 1, 3, 7, 15, 31, 63, 127, 255, 511, 1000]
    # beta = 1.5: sizes ceil((3/2)^i) computed exactly with rationals
    N = 10 ** 6
    b = oracle.batch_bounds(N, 1.5)
    want, pos, i = [0], 0, 0
    while pos < N:
        x = Fraction(3, 2) ** i
        sz = -(-x.numerator // x.denominator)
        pos = min(N, pos + sz)
        want.append(pos)
        i += 1
    assert b.tolist() == want
    assert oracle.batch_bounds(0, 1.5).tolist() == [0]
    assert oracle.batch_bounds(1, 1.5).tolist() == [0, 1]


def test_pivot_order_is_a_seeded_bijection():
    rng = np.random.default_rng(5)
    for n in (1, 2, 3, 5, 64, 1000, 4097):
        active = (rng.random(n) < 0.7).astype(np.uint8)
        o1 = oracle.pivot_order(active, seed=42)
        assert np.array_equal(np.sort(o1), np.flatnonzero(active))
        assert np.array_equal(o1, oracle.pivot_order(active, seed=42))
        if active.sum() > 20:
            o2 = oracle.pivot_order(active, seed=43)
            assert not np.array_equal(o1, o2)
            assert not np.array_equal(o1, np.flatnonzero(active))


def test_pivot_round_function_is_splitmix64():
    """The round function is the SplitMix64 finaliser (Steele, Lea & Flood,
    OOPSLA 2014). The generator adds 0x9E3779B97F4A7C15 to its state and returns
    the finaliser of the new state; from state 1234567 its published reference
    implementation (Vigna's splitmix64.c) gives the five outputs below."""
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
            16408922859458223821]
    state, got = 1234567, []
    for _ in want:
        state = (state + 0x9E3779B97F4A7C15) % 2**64
        got.append(oracle.mix64(state))
    assert got == want


# ------------------------------------------------- the method's own steps --

def test_bgss_model_reaches_the_scc_partition():
    """The sequential model of Alg. 1 with the library's readings (trim once,
    first SCC, class trimming, prefix-doubling batches, classes by (old class,
    max forward source, max backward source), canonical minimum) gives Tarjan's
    labels: on every digraph with 3 vertices (self-loops included), on random
    digraphs for several beta and pivot seeds, with and without class trimming."""
    from oracle.bgss_model import bgss_labels
    for edges in _all_digraphs(3, True):
        off, adj = _csr(3, edges)
        lab, _ = bgss_labels(3, off, adj)
        assert np.array_equal(lab, oracle.scc_labels(3, off, adj)[0]), edges
    rng = np.random.default_rng(0xB655)
    for trial in range(400):
        n = int(rng.integers(1, 61))
        g = gg.gnp(n, float(rng.choice([0.02, 0.05, 0.1, 0.3])), seed=9000 + trial, allow_self=trial % 4 == 0)
        want, _ = oracle.scc_labels(n, g.offsets, g.targets)
        beta = float(rng.choice([1.1, 1.5, 2.0, 3.0]))
        lab, st = bgss_labels(n, g.offsets, g.targets, beta=beta, seed=int(rng.integers(1 << 62)),
                              class_trim=bool(trial % 2))
        assert np.array_equal(lab, want), (trial, n, beta)
        assert st["n_trimmed"] == int(oracle.trim(n, g.offsets, g.targets).sum())


def test_bgss_model_with_the_batched_kernels_cut_reaches_the_scc_partition():
    """Reading r17 (the batched kernel's cut of the pivot order: further
    single-pivot steps while a step leaves 1/8 of the active vertices reached
    one way only, batches after those positions, and a small batch whose pairs
    pass a cap taken one pivot at a time) still gives Tarjan's labels: on every
    digraph with 3 vertices, on random digraphs and on tori, R-MAT and k-NN
    graphs, with pair caps small enough that the per-source fallback runs."""
    from oracle.bgss_model import bgss_labels
    r17 = dict(single_steps=8, single_fallback=16)
    for edges in _all_digraphs(3, True):
        off, adj = _csr(3, edges)
        lab, _ = bgss_labels(3, off, adj, pair_cap=1, **r17)
        assert np.array_equal(lab, oracle.scc_labels(3, off, adj)[0]), edges
    rng = np.random.default_rng(0xB617)
    steps = fallbacks = 0
    for trial in range(300):
        n = int(rng.integers(1, 61))
        g = gg.gnp(n, float(rng.choice([0.02, 0.05, 0.1, 0.3])), seed=9400 + trial, allow_self=trial % 4 == 0)
        want, _ = oracle.scc_labels(n, g.offsets, g.targets)
        lab, st = bgss_labels(n, g.offsets, g.targets, beta=float(rng.choice([1.5, 2.0, 3.0])),
                              seed=int(rng.integers(1 << 62)), pair_cap=int(rng.integers(0, 40)), **r17)
        assert np.array_equal(lab, want), (trial, n)
        steps += st["single_steps"] - 1
        fallbacks += st["fallback_batches"]
    for g in (gg.torus(2, 16, 0.5, seed=3), gg.torus(3, 6, 0.4, seed=4), gg.rmat(9, 4, seed=5),
              gg.knn(400, 3, seed=6)):
        want, _ = oracle.scc_labels(g.n, g.offsets, g.targets)
        for cap in (0, 8, 64):
            lab, st = bgss_labels(g.n, g.offsets, g.targets, pair_cap=cap, **r17)
            assert np.array_equal(lab, want), (g.n, cap)
            steps += st["single_steps"] - 1
            fallbacks += st["fallback_batches"]
    assert steps > 0 and fallbacks > 0  # both parts of the reading ran


@pytest.mark.parametrize("make", [lambda: gg.torus(2, 16, 0.5, seed=3), lambda: gg.torus(3, 6, 0.4, seed=4),
                                  lambda: gg.rmat(9, 4, seed=5), lambda: gg.knn(400, 3, seed=6)])
def test_bgss_model_on_structured_graphs(make):
    from oracle.bgss_model import bgss_labels
    g = make()
    want, _ = oracle.scc_labels(g.n, g.offsets, g.targets)
    lab, st = bgss_labels(g.n, g.offsets, g.targets)
    assert np.array_equal(lab, want)
    # the first SCC is the SCC of the first pivot of the seeded order
    active = 1 - oracle.trim(g.n, g.offsets, g.targets)
    order = oracle.pivot_order(active, seed=0x5CC00)
    assert st["first_scc_size"] == (int((want == want[order[0]]).sum()) if len(order) else 0)
