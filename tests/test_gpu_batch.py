"""Batched SCC (include/scc_batch.h): every graph of a packed batch gets the
labels the CPU oracle (iterative Tarjan) gives it alone, for several kernel
configurations, on CUDA-graph replays, with host and device output, and under
the autotuner's choice."""
import numpy as np
import pytest

import oracle
from paper_2303_04934_gb300 import graphgen as gg
from paper_2303_04934_gb300 import scc

from gpu_util import dev, ensure_lib

pytestmark = pytest.mark.gpu


def _edge_graphs():
    yield gg.from_edges(0, [], name="empty")
    yield gg.from_edges(1, [], name="one_vertex")
    yield gg.from_edges(1, [(0, 0)], name="self_loop")
    yield gg.from_edges(5, [(i, (i + 1) % 5) for i in range(5)], name="cycle5")
    yield gg.from_edges(6, [(i, i + 1) for i in range(5)], name="path6")
    yield gg.from_edges(4, [(a, b) for a in range(4) for b in range(4) if a != b], name="complete4")
    yield gg.from_edges(6, [(0, 1), (1, 2), (2, 0), (3, 4), (4, 5), (5, 3), (2, 3), (2, 3)], name="two_cycles_dup")


def _batch():
    gs = list(_edge_graphs())
    gs += [gg.gnp(80, 0.03, seed=900 + i, allow_self=i % 2 == 0) for i in range(6)]
    gs += [gg.torus(2, s, 0.5, seed=910 + s) for s in (8, 23, 40, 64)]
    gs += [gg.rmat(s, 8, seed=920 + s) for s in (6, 9, 12, 14)]
    gs += [gg.torus(3, 12, 0.3, seed=930), gg.knn(3000, 5, seed=931)]
    # deep and skewed structures: a long path and a long cycle (ids shuffled),
    # a star with a 20k-arc hub in both directions, a chain of small cliques
    rng = np.random.default_rng(940)
    p = rng.permutation(8000)
    gs.append(gg.from_edges(8000, [(int(p[i]), int(p[i + 1])) for i in range(7999)], name="path8k"))
    gs.append(gg.from_edges(8000, [(int(p[i]), int(p[(i + 1) % 8000])) for i in range(8000)], name="cycle8k"))
    k = 20000
    gs.append(gg.from_edges(k, [(0, i) for i in range(1, k)] + [(i, 0) for i in range(1, k, 3)], name="star20k"))
    e = []
    for c in range(500):
        e += [(4 * c + x, 4 * c + y) for x in range(4) for y in range(4) if x != y]
        if c < 499:
            e.append((4 * c + 3, 4 * c + 4))
    gs.append(gg.from_edges(2000, e, name="clique_chain"))
    return gg.pack(gs)


_PACKED = None


def packed():
    global _PACKED
    if _PACKED is None:
        _PACKED = _batch()
    return _PACKED


def _expect(p):
    return [oracle.scc_labels(p.graph(g).n, p.graph(g).offsets, p.graph(g).targets)[0] for g in range(p.G)]


_WANT = None


def want():
    global _WANT
    if _WANT is None:
        _WANT = _expect(packed())
    return _WANT


def _check(p, labels):
    for g, w in enumerate(want()):
        got = p.labels_of(labels, g)
        assert np.array_equal(got, w), (g, p.names[g])


def _cfg(**kw):
    c = scc.scc_batch_config_default()
    for k, v in kw.items():
        setattr(c, "lambda_" if k == "lam" else k, v)
    return c


@pytest.mark.parametrize("kw", [dict(), dict(tau=16, block=128, lam=1024), dict(tau=4096, block=512, lam=65536),
                                dict(tau=64, block=256, seeds=4, beta=1.5), dict(seed=777, beta=3.0),
                                dict(blocks_per_sm=1)])
def test_batch_labels_match_oracle(kw):
    import torch
    ensure_lib()
    p = packed()
    with scc.SccBatch(p, config=_cfg(**kw)) as B:
        out = torch.full((int(p.vbase[-1]),), -7, dtype=torch.int32, device="cuda")
        B.labels(out)
        torch.cuda.synchronize()
        _check(p, out.cpu().numpy())
        # a second run replays the captured graph and must give the same labels
        out2 = torch.full_like(out, -9)
        B.labels(out2)
        B.labels(out2)
        torch.cuda.synchronize()
        assert torch.equal(out, out2)
        st = B.stats()
        assert st["graphs"] == p.G and st["replays"] == 3 and st["captures"] == 2


def test_batch_host_buffers_and_device_input():
    ensure_lib()
    p = packed()
    dp = gg.Packed(p.G, dev(p.vbase), dev(p.ebase), dev(p.offsets), dev(p.targets), p.names)
    with scc.SccBatch(dp) as B:
        out = np.full(int(p.vbase[-1]), -3, np.int32)
        scc.scc_batch_run(B.h, out)
        _check(p, out)


def test_batch_mixed_generator_and_autotune():
    import torch
    ensure_lib()
    p = gg.mixed_batch(24, 1000, 30000, seed=4242)
    want_l = [oracle.scc_labels(p.graph(g).n, p.graph(g).offsets, p.graph(g).targets)[0] for g in range(p.G)]
    with scc.SccBatch(p) as B:
        start = scc.scc_batch_get_config(B.h)
        best, ms = scc.scc_batch_autotune(B.h, sample=6)
        # the tuner keeps the handle's configuration unless a grid point beats it
        kept = (best.tau, best.block, best.lambda_) == (start.tau, start.block, start.lambda_)
        assert ms > 0 and (kept or (best.block in (128, 256, 512, 1024) and best.tau in (16, 64, 256, 1024, 4096)
                                    and best.lambda_ in (256, 1024, 4096, 16384)))
        got = scc.scc_batch_get_config(B.h)
        assert (got.tau, got.block, got.lambda_) == (best.tau, best.block, best.lambda_)
        out = B.labels()
        torch.cuda.synchronize()
        lab = out.cpu().numpy()
        for g in range(p.G):
            assert np.array_equal(p.labels_of(lab, g), want_l[g]), g


def test_batch_precomputed_transpose_spans_groups():
    """The G^T computed before the launch is built for groups of consecutive
    graphs of at most 2^24 vertices: 18 graphs of 10^6 vertices make two
    groups (and an empty graph and a self-loop graph sit inside them). The
    graphs at the group boundary and at both ends are checked."""
    import torch
    ensure_lib()
    gs = [gg.torus(2, 1000, 0.5, seed=950 + i) for i in range(18)]
    gs.insert(7, gg.from_edges(0, [], name="empty"))
    gs.insert(12, gg.from_edges(3, [(0, 0), (0, 1), (1, 0), (2, 2)], name="self_loops"))
    p = gg.pack(gs)
    with scc.SccBatch(p) as B:
        out = B.labels()
        torch.cuda.synchronize()
        lab = out.cpu().numpy()
    for g in (0, 7, 12, 16, 17, 18, 19):
        want, _ = oracle.scc_labels(p.graph(g).n, p.graph(g).offsets, p.graph(g).targets)
        assert np.array_equal(p.labels_of(lab, g), want), g


def test_batch_rejects_malformed_input():
    ensure_lib()
    g = gg.from_edges(3, [(0, 1), (1, 2)])
    bad = gg.Graph(3, g.offsets, np.array([0, 5], np.int32))  # target out of range
    p = gg.pack([g, bad])
    with pytest.raises(scc.SccError) as e:
        scc.scc_batch_create(p.G, p.vbase, p.ebase, p.offsets, p.targets)
    assert e.value.code == scc.SCC_ERR_INVALID_ARG
    vb = p.vbase.copy()
    vb[1] = 7  # vertex bases inconsistent with the offsets
    with pytest.raises(scc.SccError):
        scc.scc_batch_create(p.G, vb, p.ebase, p.offsets, p.targets)
    with pytest.raises(scc.SccError):
        h = scc.scc_batch_create(p.G - 1, p.vbase[:2], p.ebase[:2], p.offsets[:4], p.targets[:2])
        c = _cfg(block=100)
        try:
            scc.scc_batch_set_config(h, c)
        finally:
            scc.scc_batch_destroy(h)


def test_batch_empty():
    ensure_lib()
    p = gg.pack([])
    h = scc.scc_batch_create(0, p.vbase, p.ebase, p.offsets, p.targets)
    scc.scc_batch_run(h, np.zeros(1, np.int32))
    scc.scc_batch_destroy(h)


def _cycle_chain(L: int, k: int, seed: int, name: str):
    """L k-cliques in a line (clique c -> clique c+1 by one arc), vertex ids
    shuffled: L SCCs, each reaching every clique after it, so a few sources
    fill a batch's pair tables."""
    rng = np.random.default_rng(seed)
    p = rng.permutation(L * k)
    e = []
    for c in range(L):
        e += [(int(p[k * c + x]), int(p[k * c + y])) for x in range(k) for y in range(k) if x != y]
        if c + 1 < L:
            e.append((int(p[k * c + k - 1]), int(p[k * c + k])))
    return gg.from_edges(L * k, e, name=name)


def test_batch_overflowing_batches_take_single_pivot_steps():
    """Chains of SCCs where every source reaches a long stretch of the chain:
    batches overflow their pair tables, small ones are then taken one pivot at
    a time and larger ones rerun with bigger tables or fewer sources. Labels
    match the oracle, on the lattice-like path (2-cycles) and on the dense one
    (10-cliques: 9 arcs per vertex, forward and backward searches apart)."""
    import torch
    ensure_lib()
    gs = [_cycle_chain(3000, 2, 960, "chain2x3000"), _cycle_chain(50000, 2, 961, "chain2x50000"),
          _cycle_chain(2000, 10, 962, "chain10x2000")]
    p = gg.pack(gs)
    with scc.SccBatch(p) as B:
        out = B.labels()
        torch.cuda.synchronize()
        lab = out.cpu().numpy()
        t = scc.scc_debug_batch_times(B.h, p.G)
    for g in range(p.G):
        want, _ = oracle.scc_labels(p.graph(g).n, p.graph(g).offsets, p.graph(g).targets)
        assert np.array_equal(p.labels_of(lab, g), want), p.names[g]
    assert t[1, 9] > 0, "the long chain reran a batch"
