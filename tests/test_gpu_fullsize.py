"""GPU labels at the full configuration sizes, in the configuration bench.py
times (default scc_config, device-resident CSR, labels to device memory),
compared element by element with the CPU oracle (iterative Tarjan for SCCs,
union-find for connected components):

* R-MAT scale 24, edge factor 16 (the benchmark workload),
* 3D torus 256^3 with every arc present with p = 0.3,
* directed 5-NN graph of 8 M points from 64 Gaussians (sigma 0.02);

and the least-element lists of R-MAT scale 20 (the size bench.py times them
at) against the oracle's sequential pruned BFS for the same order.
"""
import numpy as np
import pytest

import oracle
from paper_2303_04934_gb300 import graphgen as gg
from paper_2303_04934_gb300 import scc

from gpu_util import ensure_lib, labels_of, make_graph

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("make", [
    lambda: gg.rmat(24, 16, seed=0x5CC01),
    lambda: gg.torus(3, 256, 0.3, seed=0x5CC02),
    lambda: gg.knn(8_000_000, 5, seed=0x5CC03),
], ids=["rmat24", "torus3d_256", "knn8m"])
def test_full_size_labels_match_tarjan(make):
    ensure_lib()
    g = make()
    want, nscc = oracle.scc_labels(g.n, g.offsets, g.targets)
    with make_graph(g) as G:
        got = labels_of(G)
        st = G.stats()
        import torch
        cc = torch.empty(g.n, dtype=torch.int32, device="cuda")
        scc.cc_run(G.h, cc)
        torch.cuda.synchronize()
        cc = cc.cpu().numpy()
    assert np.array_equal(got, want)
    assert st["n_trimmed"] <= nscc
    want_cc, _ = oracle.cc_labels(g.n, g.offsets, g.targets)
    assert np.array_equal(cc, want_cc)
    assert np.array_equal(cc[got], cc)  # every SCC lies inside one component


def test_le_lists_rmat20_match_sequential():
    import torch
    ensure_lib()
    g = gg.rmat(20, 16, seed=0x5CC01)
    with make_graph(g) as G:
        total = scc.le_lists_run(G.h)
        order = torch.empty(g.n, dtype=torch.int32, device="cuda")
        off = torch.empty(g.n + 1, dtype=torch.int64, device="cuda")
        src = torch.empty(max(total, 1), dtype=torch.int32, device="cuda")
        dist = torch.empty(max(total, 1), dtype=torch.int32, device="cuda")
        scc.le_lists_get(G.h, order, off, src[:total], dist[:total], total)
        torch.cuda.synchronize()
    order = order.cpu().numpy()
    w_off, w_src, w_dist = oracle.le_lists(g.n, g.offsets, g.targets, order)
    assert np.array_equal(off.cpu().numpy(), w_off)
    assert np.array_equal(src.cpu().numpy()[:total], w_src)
    assert np.array_equal(dist.cpu().numpy()[:total], w_dist)
