"""GPU labels at the full configuration sizes, in the configuration bench.py
times (default scc_config, device-resident CSR, labels to device memory),
compared element by element with the CPU oracle (iterative Tarjan):

* R-MAT scale 24, edge factor 16 (the benchmark workload),
* 3D torus 256^3 with every arc present with p = 0.3,
* directed 5-NN graph of 8 M points from 64 Gaussians (sigma 0.02).
"""
import numpy as np
import pytest

import oracle
from paper_2303_04934_gb300 import graphgen as gg

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
    assert np.array_equal(got, want)
    assert st["n_trimmed"] <= nscc
