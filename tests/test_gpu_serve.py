"""Serving (include/scc_serve.h): every request gets the same result alone and
in a mix of concurrent requests (continuous batching: batched SCC launches,
merged reachability launches, the full-GPU path), equal to the CPU oracle;
admission respects the memory cap; malformed requests are refused."""
import numpy as np
import pytest

import oracle
from paper_2303_04934_gb300 import graphgen as gg
from paper_2303_04934_gb300 import scc

from gpu_util import ensure_lib

pytestmark = pytest.mark.gpu


def _graphs():
    return [gg.torus(2, 30, 0.5, seed=601), gg.rmat(10, 8, seed=602), gg.gnp(200, 0.02, seed=603, allow_self=True),
            gg.torus(3, 14, 0.3, seed=604), gg.rmat(14, 8, seed=605), gg.torus(2, 90, 0.5, seed=606),
            gg.from_edges(1, [(0, 0)]), gg.from_edges(4, [(0, 1), (1, 2), (2, 3)]), gg.knn(5000, 5, seed=607)]


RESIDENT = None


def _resident():
    global RESIDENT
    if RESIDENT is None:
        RESIDENT = [gg.torus(2, 64, 0.5, seed=611), gg.rmat(12, 8, seed=612)]
    return RESIDENT


def _requests(rng):
    """(kind, args) list: SCC requests on the pool graphs, reach queries on the
    resident graphs (several on the same graph and direction, so they merge)."""
    reqs = [("scc", i) for i in range(len(_graphs()))] * 2
    for _ in range(24):
        gi = int(rng.integers(0, 2))
        n = _resident()[gi].n
        k = int(rng.integers(1, 49))  # merged launches pass 64 sources (two mask words)
        reqs.append(("reach", gi, rng.integers(0, n, k).astype(np.int32), int(rng.integers(0, 2))))
    order = rng.permutation(len(reqs))
    return [reqs[i] for i in order]


def _run(srv, gids, reqs, together):
    pool = _graphs()
    outs, rids = [], []
    for r in reqs:
        if r[0] == "scc":
            g = pool[r[1]]
            out = np.full(g.n, -5, np.int32)
            rid = srv.submit_scc(g.n, np.ascontiguousarray(g.offsets), np.ascontiguousarray(g.targets), out)
        else:
            g = _resident()[r[1]]
            out = np.zeros(g.n, np.uint64)
            rid = srv.submit_reach(gids[r[1]], r[2], r[3], out)
        outs.append(out)
        if together:
            rids.append(rid)
        else:
            st, _ = srv.wait(rid)
            assert st == scc.SCC_OK
    for rid in rids:
        st, lat = srv.wait(rid)
        assert st == scc.SCC_OK and lat >= 0
    return outs


def _expect(r):
    if r[0] == "scc":
        g = _graphs()[r[1]]
        return oracle.scc_labels(g.n, g.offsets, g.targets)[0]
    g = _resident()[r[1]]
    if r[3] == 0:
        return oracle.reach_mask(g.n, g.offsets, g.targets, r[2])
    toff, tadj = oracle.transpose(g.n, g.offsets, g.targets)
    return oracle.reach_mask(g.n, toff, tadj, r[2])


@pytest.mark.parametrize("mode", ["batched_merged", "plain_only"])
def test_serve_alone_equals_mix_equals_oracle(mode):
    ensure_lib()
    cfg = scc.scc_server_config_default()
    if mode == "batched_merged":
        cfg.batch_vertices = 8192  # the two largest pool graphs take the full-GPU path
    else:
        cfg.batch_vertices = 0
        cfg.merge_reach = 0
        cfg.prefetch = 0
    rng = np.random.default_rng(77)
    reqs = _requests(rng)
    with scc.SccServer(cfg) as srv:
        gids = [srv.add_graph(g.n, np.ascontiguousarray(g.offsets), np.ascontiguousarray(g.targets))
                for g in _resident()]
        alone = _run(srv, gids, reqs, together=False)
        srv.reset_stats()
        mix = _run(srv, gids, reqs, together=True)
        st = srv.stats()
    for r, a, b in zip(reqs, alone, mix):
        assert np.array_equal(a, b), r[:2]
        assert np.array_equal(a, _expect(r)), r[:2]
    assert st["completed"] == len(reqs) and st["failed"] == 0
    if mode == "batched_merged":
        assert st["batched_launches"] >= 1 and st["batched_graphs"] > st["batched_launches"]
        assert st["plain_scc"] >= 1
        assert st["reach_shared"] >= 2 and st["reach_launches"] < st["reach_requests"]
    else:
        assert st["batched_launches"] == 0 and st["reach_shared"] == 0
        assert st["plain_scc"] == st["scc_requests"]


def test_serve_memory_cap_admission():
    ensure_lib()
    big = gg.rmat(15, 8, seed=621)
    cfg = scc.scc_server_config_default()
    cfg.batch_vertices = 0
    # room for about two full-GPU requests of this size at a time
    per = 18 * big.m + 360 * big.n + (64 << 20)
    cfg.mem_cap_bytes = int(2.5 * per)
    want = oracle.scc_labels(big.n, big.offsets, big.targets)[0]
    with scc.SccServer(cfg) as srv:
        outs = [np.full(big.n, -1, np.int32) for _ in range(6)]
        rids = [srv.submit_scc(big.n, big.offsets, big.targets, o) for o in outs]
        for rid in rids:
            assert srv.wait(rid)[0] == scc.SCC_OK
        st = srv.stats()
        assert st["mem_peak"] <= cfg.mem_cap_bytes and st["max_admitted"] <= 2
        for o in outs:
            assert np.array_equal(o, want)
        # a request larger than the cap alone is refused at once
        huge = gg.rmat(19, 8, seed=622)
        assert 18 * huge.m + 360 * huge.n + (64 << 20) > cfg.mem_cap_bytes
        with pytest.raises(scc.SccError) as e:
            srv.submit_scc(huge.n, huge.offsets, huge.targets, np.zeros(huge.n, np.int32))
        assert e.value.code == scc.SCC_ERR_OOM


def test_serve_rejects_bad_requests():
    ensure_lib()
    g = gg.torus(2, 8, 0.5, seed=631)
    with scc.SccServer() as srv:
        gid = srv.add_graph(g.n, g.offsets, g.targets)
        out = np.zeros(g.n, np.uint64)
        for args in [(gid + 7, [0], 0), (gid, [0] * 65, 0), (gid, [g.n], 0), (gid, [0], 2)]:
            with pytest.raises(scc.SccError) as e:
                srv.submit_reach(args[0], np.array(args[1], np.int32), args[2], out)
            assert e.value.code == scc.SCC_ERR_INVALID_ARG
        # an SCC request whose graph is malformed completes with an error status
        bad = np.array([0, 5], np.int32)
        rid = srv.submit_scc(2, np.array([0, 1, 2], np.int32), bad, np.zeros(2, np.int32))
        assert srv.wait(rid)[0] == scc.SCC_ERR_INVALID_ARG
        rid = srv.submit_reach(gid, np.array([1, 2], np.int32), 1, out)
        srv.drain()
        srv.remove_graph(gid)
        assert srv.stats()["resident_graphs"] == 0
