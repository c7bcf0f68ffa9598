"""The serving loop's scheduling decisions (admission under the memory cap,
the requests that form a dispatch unit), called through the C ABI on the host:
hand-made queues with known answers, and random queues against a model of the
rules include/scc_serve.h states. CPU only."""
import numpy as np
import pytest

from paper_2303_04934_gb300 import scc

MB = 1 << 20


def _admission_model(need, waited, in_use, cap, max_bypass):
    taken, blocked = [], False
    for i, (nd, w) in enumerate(zip(need, waited)):
        if in_use + nd <= cap:
            taken.append(i)
            in_use += nd
        elif not blocked and w > max_bypass:
            break
        else:
            blocked = True
    return taken


def _unit_model(kind, small, graph, dir_, nsrc, merge, batch_graphs, batch_min=1):
    if not kind:
        return []
    if kind[0] == 1:
        out, k = [], 0
        for i in range(len(kind)):
            same = kind[i] == 1 and graph[i] == graph[0] and dir_[i] == dir_[0]
            if same and (not out or (merge and k + nsrc[i] <= 128)):
                out.append(i)
                k += nsrc[i]
            if not merge:
                break
        return out
    if small[0]:
        smalls = [i for i in range(len(kind)) if kind[i] == 0 and small[i]]
        return smalls[:batch_graphs] if len(smalls) >= batch_min else [0]
    return [0]


def test_admission_hand_cases():
    f = scc.scc_debug_serve_admission
    # everything fits: all, in order
    assert f([1, 2, 3], [0, 0, 0], 0, 10, 50.0) == [0, 1, 2]
    # the cap is reached: a later small request passes a large one that has not waited long
    assert f([6, 6, 2], [0, 0, 0], 0, 10, 50.0) == [0, 2]
    # ... but not once the large one has waited longer than max_bypass_ms
    assert f([6, 6, 2], [0, 60, 0], 0, 10, 50.0) == [0]
    # only the first request that does not fit can stop the pass
    assert f([6, 6, 6, 2], [0, 10, 90, 0], 0, 10, 50.0) == [0, 3]
    # bytes already in use count; equality with the cap fits
    assert f([4, 1], [0, 0], 6, 10, 50.0) == [0]
    assert f([4, 1], [0, 0], 5, 10, 50.0) == [0, 1]
    # nothing pending
    assert f([], [], 0, 10, 50.0) == []
    with pytest.raises(scc.SccError):
        f([-1], [0], 0, 10, 50.0)


def test_admission_random_queues_match_the_rule():
    rng = np.random.default_rng(0x5E7)
    for trial in range(3000):
        count = int(rng.integers(0, 40))
        need = rng.integers(0, 64, count) * MB
        waited = rng.uniform(0, 100, count)
        in_use = int(rng.integers(0, 128)) * MB
        cap = int(rng.integers(64, 512)) * MB
        bypass = float(rng.choice([0.0, 10.0, 50.0, 1e9]))
        want = _admission_model(need.tolist(), waited.tolist(), in_use, cap, bypass)
        assert scc.scc_debug_serve_admission(need, waited, in_use, cap, bypass) == want, trial


def test_unit_hand_cases():
    f = scc.scc_debug_serve_unit
    # reach queries on graph 3 forward merge up to 128 sources; other graphs/directions wait
    kind = [1, 1, 1, 0, 1, 1]
    small = [0, 0, 0, 1, 0, 0]
    graph = [3, 3, 4, 0, 3, 3]
    dir_ = [0, 1, 0, 0, 0, 0]
    nsrc = [64, 64, 8, 0, 60, 4]
    assert f(kind, small, graph, dir_, nsrc) == [0, 4, 5]
    # a query that would exceed 128 sources is skipped, a later smaller one joins
    assert f([1, 1, 1], [0, 0, 0], [1, 1, 1], [0, 0, 0], [100, 40, 28]) == [0, 2]
    # without merging: the oldest query alone
    assert f(kind, small, graph, dir_, nsrc, merge_reach=False) == [0]
    # small SCC requests share a batched launch, batch_graphs at most, skipping large ones and queries
    kind = [0, 0, 1, 0, 0, 0]
    small = [1, 0, 0, 1, 1, 1]
    z = [0] * 6
    assert f(kind, small, z, z, z, batch_graphs=3) == [0, 3, 4]
    # a large SCC request runs alone
    assert f([0, 0, 0], [0, 1, 1], [0] * 3, [0] * 3, [0] * 3) == [0]
    assert f([], [], [], [], []) == []


def test_unit_needs_batch_min_small_requests_for_a_batched_launch():
    f = scc.scc_debug_serve_unit
    kind, small, z = [0, 0, 1, 0], [1, 1, 0, 1], [0, 0, 0, 0]
    assert f(kind, small, z, z, [0, 0, 5, 0], batch_min=3) == [0, 1, 3]
    assert f(kind, small, z, z, [0, 0, 5, 0], batch_min=4) == [0]  # too few: the oldest alone


@pytest.mark.parametrize("merge", [True, False])
def test_unit_random_queues_match_the_rule(merge):
    rng = np.random.default_rng(0x0417 + merge)
    for trial in range(3000):
        count = int(rng.integers(1, 30))
        kind = rng.integers(0, 2, count)
        small = rng.integers(0, 2, count) * (kind == 0)
        graph = rng.integers(0, 3, count)
        dir_ = rng.integers(0, 2, count)
        nsrc = rng.integers(1, 65, count) * (kind == 1)
        bg = int(rng.integers(1, 8))
        bm = int(rng.integers(1, bg + 1))
        want = _unit_model(kind.tolist(), small.tolist(), graph.tolist(), dir_.tolist(), nsrc.tolist(), merge, bg, bm)
        got = scc.scc_debug_serve_unit(kind, small, graph, dir_, nsrc, merge_reach=merge, batch_graphs=bg,
                                       batch_min=bm)
        assert got == want, trial
        assert got[0] == 0 and got == sorted(set(got))
