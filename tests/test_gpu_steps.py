"""GPU parity of the individual hot-path steps against the CPU oracle:
CSR / transposed-CSR build (a1), trimming (a2), pivot order (a3), hash bag (a6),
pair table (a7), single-reachability (a4), multi-reachability (a5) and
reach_multi (a10). All exact (integer work)."""
import numpy as np
import pytest

import oracle
from paper_2303_04934_gb300 import graphgen as gg
from paper_2303_04934_gb300 import scc

from gpu_util import config, dev, ensure_lib, make_graph, self_loop_free, sorted_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _graphs():
    yield gg.gnp(1, 0.0, seed=1)
    yield gg.from_edges(3, [], name="no_arcs")
    yield gg.from_edges(4, [(0, 0), (1, 1), (1, 2), (2, 1), (3, 3), (3, 3)], name="self_loops")
    yield gg.gnp(60, 0.08, seed=2, allow_self=True)
    yield gg.gnp(300, 0.01, seed=3, allow_self=True)
    yield gg.torus(2, 33, 0.5, seed=4)
    yield gg.torus(3, 12, 0.3, seed=5)
    yield gg.rmat(14, 8, seed=6)
    yield gg.knn(20000, 5, seed=7)
    yield gg.rmat(20, 16, seed=8)  # ~40% empty rows: row searches end on empty rows


@pytest.mark.parametrize("g", list(_graphs()), ids=lambda g: g.name)
def test_csr_transpose_and_trim(g):
    import torch
    with make_graph(g) as G:
        n, m, mt = scc.scc_graph_info(G.h)
        off0, adj0 = self_loop_free(g)
        assert (n, m, mt) == (g.n, g.m, len(adj0))
        off = np.empty(n + 1, np.int32)
        adj = np.empty(max(mt, 1), np.int32)
        scc.scc_debug_csr(G.h, 0, off, adj)
        assert np.array_equal(off, off0) and np.array_equal(adj[:mt], adj0)
        toff_o, tadj_o = oracle.transpose(g.n, g.offsets, g.targets)
        scc.scc_debug_csr(G.h, 1, off, adj)
        assert np.array_equal(off, toff_o)
        assert np.array_equal(sorted_rows(off, adj[:mt]), tadj_o)  # oracle rows are increasing
        fl = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
        scc.scc_debug_trim(G.h, fl)
        torch.cuda.synchronize()
        assert np.array_equal(fl.cpu().numpy()[:n], oracle.trim(g.n, g.offsets, g.targets))


def test_invalid_csr_rejected():
    ensure_lib()
    bad = [
        (3, np.array([0, 1, 2, 2], np.int32), np.array([0, 5], np.int32)),   # target out of range
        (3, np.array([0, 2, 1, 2], np.int32), np.array([0, 1], np.int32)),   # offsets decrease
        (3, np.array([1, 1, 2, 2], np.int32), np.array([0, 1], np.int32)),   # offsets[0] != 0
        (2, np.array([0, 1, 1], np.int32), np.array([-1], np.int32)),        # negative target
    ]
    for n, off, adj in bad:
        with pytest.raises(scc.SccError) as e:
            scc.scc_graph_create(n, len(adj), dev(off), dev(adj))
        assert e.value.code == scc.SCC_ERR_INVALID_ARG


@pytest.mark.parametrize("seed", [0x5CC00, 1, 2**63 + 5])
def test_pivot_order_bit_exact(seed):
    g = gg.rmat(13, 4, seed=11)
    with make_graph(g, config(seed=seed)) as G:
        order = np.empty(g.n, np.int32)
        N = scc.scc_debug_pivot_order(G.h, order)
        active = 1 - oracle.trim(g.n, g.offsets, g.targets)
        want = oracle.pivot_order(active, seed)
        assert N == len(want) and np.array_equal(order[:N], want)


@pytest.mark.parametrize("count,lam,sigma", [(1, 1024, 50), (1000, 1024, 50), (300000, 1024, 50),
                                             (300000, 16384, 50), (1 << 21, 1024, 8)])
def test_hash_bag_extracts_the_inserted_multiset(count, lam, sigma):
    rng = np.random.default_rng(count)
    items = rng.integers(0, 2**31 - 2, count).astype(np.int32)
    items[: count // 3] = items[0]  # duplicates are kept (the bag does not dedupe)
    out = np.empty(count, np.int32)
    nout, chunks = scc.scc_debug_hashbag(items, count, lam, sigma, out)
    assert nout == count
    assert np.array_equal(np.sort(out), np.sort(items))
    if count >= 300000 and lam == 1024:
        assert chunks > 3  # resized on the device


@pytest.mark.parametrize("count,init_cap", [(5000, 1024), (200000, 1024), (200000, 1 << 20)])
def test_pair_table_set_semantics_and_regrowth(count, init_cap):
    rng = np.random.default_rng(count + init_cap)
    keys = (rng.integers(0, 50000, count).astype(np.uint64) << np.uint64(32)) | rng.integers(0, 64, count).astype(np.uint64)
    out = np.empty(count, np.uint64)
    nout, resizes = scc.scc_debug_pair_table(keys, count, init_cap, out)
    assert np.array_equal(np.sort(out[:nout]), np.unique(keys))
    if init_cap == 1024:
        assert resizes > 0


def _reach_cases():
    yield gg.torus(2, 40, 0.5, seed=21)
    yield gg.torus(3, 14, 0.35, seed=22)
    yield gg.rmat(13, 8, seed=23)
    yield gg.knn(8000, 5, seed=24)
    yield gg.gnp(200, 0.02, seed=25, allow_self=True)


@pytest.mark.parametrize("tau,seeds", [(512, 32), (1, 1), (16, 8), (4096, 32)])
@pytest.mark.parametrize("g", list(_reach_cases()), ids=lambda g: g.name)
def test_single_reach(g, tau, seeds):
    rng = np.random.default_rng(g.n + tau)
    toff, tadj = oracle.transpose(g.n, g.offsets, g.targets)
    with make_graph(g, config(tau=tau, seeds=seeds)) as G:
        labels = rng.integers(-1, 2, g.n).astype(np.int32)
        for s in rng.integers(0, g.n, 3):
            for lab in (None, labels):
                for d in (0, 1):
                    vis = np.empty(g.n, np.uint8)
                    scc.scc_debug_single_reach(G.h, lab, int(s), d, vis)
                    o, a = (g.offsets, g.targets) if d == 0 else (toff, tadj)
                    assert np.array_equal(vis, oracle.reach_set(g.n, o, a, int(s), lab)), (s, d, lab is None)


@pytest.mark.parametrize("tau,table_cap", [(512, 0), (1, 1024), (64, 1024), (4096, 0)])
@pytest.mark.parametrize("g", list(_reach_cases()), ids=lambda g: g.name)
def test_multi_reach_pairs(g, tau, table_cap):
    rng = np.random.default_rng(g.n * 7 + tau)
    toff, tadj = oracle.transpose(g.n, g.offsets, g.targets)
    with make_graph(g, config(tau=tau)) as G:
        for trial in range(3):
            labels = rng.integers(-1, 3 if trial else 1, g.n).astype(np.int32)
            k = int(rng.integers(1, min(g.n, 200)))
            sources = rng.choice(g.n, k, replace=trial == 2).astype(np.int32)
            for d in (0, 1):
                o, a = (g.offsets, g.targets) if d == 0 else (toff, tadj)
                want = oracle.multi_reach(g.n, o, a, labels, sources)
                cap = len(want) + 16
                pairs = np.empty(cap, np.uint64)
                npairs = scc.scc_debug_multi_reach(G.h, labels, sources, k, d, pairs, cap, table_cap)
                assert npairs == len(want)
                assert np.array_equal(np.sort(pairs[:npairs]), want), (trial, d)


@pytest.mark.parametrize("g", list(_reach_cases()), ids=lambda g: g.name)
def test_reach_multi_masks(g):
    import torch
    rng = np.random.default_rng(g.n)
    toff, tadj = oracle.transpose(g.n, g.offsets, g.targets)
    with make_graph(g) as G:
        for k in (1, 7, 64):
            src = rng.integers(0, g.n, k).astype(np.int32)
            if k == 64:
                src[1] = src[0]  # duplicate sources keep their own bits
            for d in (0, 1):
                o, a = (g.offsets, g.targets) if d == 0 else (toff, tadj)
                want = oracle.reach_mask(g.n, o, a, src)
                out = torch.empty(g.n, dtype=torch.int64, device="cuda")
                scc.reach_multi(G.h, dev(src), k, d, out)
                torch.cuda.synchronize()
                assert np.array_equal(out.cpu().numpy().view(np.uint64), want), (k, d)
                host_out = np.empty(g.n, np.uint64)
                scc.reach_multi(G.h, src, k, d, host_out)
                assert np.array_equal(host_out, want)
        with pytest.raises(scc.SccError):
            scc.reach_multi(G.h, np.array([g.n], np.int32), 1, 0, np.empty(g.n, np.uint64))
        with pytest.raises(scc.SccError):
            scc.reach_multi(G.h, np.zeros(65, np.int32), 65, 0, np.empty(g.n, np.uint64))


@pytest.mark.parametrize("tau", [0, 1, 64])
@pytest.mark.parametrize("g", list(_reach_cases()), ids=lambda g: g.name)
def test_reach_multi_wide_masks(g, tau):
    """Up to 128 sources in two mask words per vertex (the serving loop's merged
    launches): each word equals the 64-source masks of its half of the sources."""
    import torch
    rng = np.random.default_rng(g.n + 5 + tau)
    toff, tadj = oracle.transpose(g.n, g.offsets, g.targets)
    with make_graph(g, config(tau=tau)) as G:
        for k in (1, 65, 100, 128):
            src = rng.integers(0, g.n, k).astype(np.int32)
            if k > 64:
                src[64] = src[0]  # one vertex in both words
            for d in (0, 1):
                o, a = (g.offsets, g.targets) if d == 0 else (toff, tadj)
                want = np.zeros(2 * g.n, np.uint64)
                want[0::2] = oracle.reach_mask(g.n, o, a, src[:64])
                if k > 64:
                    want[1::2] = oracle.reach_mask(g.n, o, a, src[64:])
                out = np.empty(2 * g.n, np.uint64)
                scc.scc_debug_reach_multi_wide(G.h, src, k, d, out)
                assert np.array_equal(out, want), (k, d)
                out_d = torch.empty(2 * g.n, dtype=torch.int64, device="cuda")
                scc.scc_debug_reach_multi_wide(G.h, dev(src), k, d, out_d)
                torch.cuda.synchronize()
                assert np.array_equal(out_d.cpu().numpy().view(np.uint64), want), (k, d)
        with pytest.raises(scc.SccError):
            scc.scc_debug_reach_multi_wide(G.h, np.zeros(129, np.int32), 129, 0, np.empty(2 * g.n, np.uint64))
        with pytest.raises(scc.SccError):
            scc.scc_debug_reach_multi_wide(G.h, np.array([g.n], np.int32), 1, 0, np.empty(2 * g.n, np.uint64))


def test_transpose_large_vertex_count_direct_path():
    """n above 2^26 takes the direct (global-atomic) transpose path."""
    import torch
    n = (1 << 26) + 5
    rng = np.random.default_rng(99)
    m = 1 << 20
    src = np.sort(rng.integers(0, n, m))
    dst = rng.integers(0, n, m).astype(np.int32)
    off = np.zeros(n + 1, np.int32)
    np.add.at(off, src + 1, 1)
    off = np.cumsum(off).astype(np.int32)
    g = gg.Graph(n, off, dst, "sparse_huge_n")
    with make_graph(g) as G:
        _, _, mt = scc.scc_graph_info(G.h)
        toff = torch.empty(n + 1, dtype=torch.int32, device="cuda")
        tadj = torch.empty(mt, dtype=torch.int32, device="cuda")
        scc.scc_debug_csr(G.h, 1, toff, tadj)
        toff_o, tadj_o = oracle.transpose(g.n, g.offsets, g.targets)
        toff_h = toff.cpu().numpy()
        assert np.array_equal(toff_h, toff_o)
        assert np.array_equal(sorted_rows(toff_h, tadj.cpu().numpy()), tadj_o)
