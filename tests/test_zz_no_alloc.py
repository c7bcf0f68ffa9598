"""reach_multi_noalloc, the entry point for callers that cannot allocate device
memory during the call (stream capture, allocator-free loops, hosts with their
own allocator): it must return exactly what reach_multi returns, on two calls in
a row (the second finds the first call's contents in the shared fixed array),
and refuse a graph too large for its fixed working array."""
import numpy as np
import pytest

from paper_2303_04934_gb300 import graphgen as gg
from paper_2303_04934_gb300 import scc

from gpu_util import dev, ensure_lib, make_graph

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("make", [lambda: gg.torus(2, 64, 0.5, seed=71), lambda: gg.rmat(13, 8, seed=72),
                                  lambda: gg.knn(20000, 5, seed=73)], ids=["torus64", "rmat13", "knn20k"])
def test_noalloc_matches_reach_multi_on_two_calls(make):
    import torch
    ensure_lib()
    g = make()
    rng = np.random.default_rng(g.n)
    with make_graph(g) as G:
        for call, (k, d) in enumerate([(64, 0), (17, 1)]):  # two calls in a row
            src = dev(rng.integers(0, g.n, k).astype(np.int32))
            want = torch.empty(g.n, dtype=torch.int64, device="cuda")
            got = torch.full((g.n,), -1, dtype=torch.int64, device="cuda")
            scc.reach_multi(G.h, src, k, d, want)
            scc.reach_multi_noalloc(G.h, src, k, d, got)
            torch.cuda.synchronize()
            assert torch.equal(got, want), (call, k, d)


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
