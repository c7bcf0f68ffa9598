"""Host logic of the batched run's G^T groups (no GPU): consecutive graphs,
greedy, within the limits, oversized graphs left to their blocks."""
import numpy as np
import pytest

from paper_2303_04934_gb300 import scc


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2303_04934_gb300 import build
    build.build()


def _check_plan(nv, na, max_v, max_a):
    vb = np.concatenate([[0], np.cumsum(nv)]).astype(np.int64)
    eb = np.concatenate([[0], np.cumsum(na)]).astype(np.int64)
    groups = scc.scc_debug_batch_groups(vb, eb, max_v, max_a)
    G = len(nv)
    member = np.full(G, -1)
    prev_end = 0
    for k, (g0, g1) in enumerate(groups):
        assert prev_end <= g0 < g1 <= G
        prev_end = g1
        member[g0:g1] = k
        sv, sa = int(nv[g0:g1].sum()), int(na[g0:g1].sum())
        assert 0 < sv <= max_v and sa <= max_a
        assert all(nv[g] <= max_v and na[g] <= max_a for g in range(g0, g1))
    for g in range(G):
        oversize = nv[g] > max_v or na[g] > max_a
        if oversize:
            assert member[g] == -1, g
        elif nv[g] > 0:
            assert member[g] >= 0, g
    # greedy: a group stops only where the next graph would not fit (or is oversized)
    for (g0, g1) in groups:
        if g1 < G and member[g1] >= 0 and groups[member[g1]][0] == g1:
            assert nv[g0:g1 + 1].sum() > max_v or na[g0:g1 + 1].sum() > max_a
    return groups


def test_groups_random_batches():
    rng = np.random.default_rng(7)
    for trial in range(60):
        G = int(rng.integers(0, 40))
        nv = rng.integers(0, 400, G)
        na = rng.integers(0, 2000, G)
        # some empty graphs and some too large for any group
        nv[rng.random(G) < 0.1] = 0
        big = rng.random(G) < 0.08
        nv[big] = 1500
        _check_plan(nv, na, max_v=1000, max_a=5000)


def test_groups_edge_cases():
    assert _check_plan(np.zeros(0, int), np.zeros(0, int), 10, 10) == []
    assert _check_plan(np.array([0, 0]), np.array([0, 0]), 10, 10) == []        # only empty graphs
    assert _check_plan(np.array([11]), np.array([0]), 10, 10) == []            # one oversized graph
    assert _check_plan(np.array([5, 5, 5]), np.array([1, 1, 1]), 10, 10) == [(0, 2), (2, 3)]
    assert _check_plan(np.array([3, 20, 3]), np.array([1, 1, 1]), 10, 10) == [(0, 1), (2, 3)]
    assert _check_plan(np.array([3, 3]), np.array([6, 6]), 10, 10) == [(0, 1), (1, 2)]   # arcs limit
    with pytest.raises(scc.SccError):
        scc.scc_debug_batch_groups(np.array([0, 5, 3]), np.array([0, 1, 2]), 10, 10)  # decreasing bases
