"""reach_multi_noalloc, the entry point for callers that may not allocate device
memory during the call (allocator-free latency-critical loops, hosts whose
device memory belongs to their own allocator). It must return exactly what
reach_multi returns and what the oracle's plain reachability masks give, on two
calls in a row (the second finds the first call's contents in the shared fixed
array), and refuse a graph too large for its fixed working array.

The file name sorts last so that a run stopping at the first failure has run
every other test first; it also passes alone in a fresh process."""
import numpy as np
import pytest

import oracle
from paper_2303_04934_gb300 import graphgen as gg
from paper_2303_04934_gb300 import scc

from gpu_util import dev, ensure_lib, make_graph

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("make", [lambda: gg.torus(2, 64, 0.5, seed=71), lambda: gg.rmat(13, 8, seed=72),
                                  lambda: gg.knn(20000, 5, seed=73)], ids=["torus64", "rmat13", "knn20k"])
def test_noalloc_matches_reach_multi_and_the_oracle_on_two_calls(make):
    import torch
    ensure_lib()
    g = make()
    rng = np.random.default_rng(g.n)
    toff, tadj = oracle.transpose(g.n, g.offsets, g.targets)
    with make_graph(g) as G:
        for call, (k, d) in enumerate([(64, 0), (17, 1)]):  # two calls in a row
            src = rng.integers(0, g.n, k).astype(np.int32)
            o, a = (g.offsets, g.targets) if d == 0 else (toff, tadj)
            ref = oracle.reach_mask(g.n, o, a, src)
            want = torch.empty(g.n, dtype=torch.int64, device="cuda")
            got = torch.full((g.n,), -1, dtype=torch.int64, device="cuda")
            scc.reach_multi(G.h, dev(src), k, d, want)
            scc.reach_multi_noalloc(G.h, dev(src), k, d, got)
            torch.cuda.synchronize()
            assert torch.equal(got, want), (call, k, d)
            assert np.array_equal(got.cpu().numpy().view(np.uint64), ref), (call, k, d)


def test_noalloc_rejects_a_graph_beyond_its_fixed_array():
    import torch
    ensure_lib()
    g = gg.torus(2, 1024, 0.5, seed=74)  # about a million vertices: more than the array holds
    with make_graph(g) as G:
        out = torch.empty(g.n, dtype=torch.int64, device="cuda")
        with pytest.raises(scc.SccError) as e:
            scc.reach_multi_noalloc(G.h, dev(np.zeros(1, np.int32)), 1, 0, out)
        assert e.value.code == scc.SCC_ERR_INVALID_ARG
        # host buffers are refused as well (the call may not stage copies)
        with pytest.raises(scc.SccError):
            scc.reach_multi_noalloc(G.h, np.zeros(1, np.int32), 1, 0, out)
