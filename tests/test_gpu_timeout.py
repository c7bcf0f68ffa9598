"""The bounded device wait behind SCC_ERR_TIMEOUT: the grid barrier that
separates the rounds of every cooperative search gives up after its limit
instead of hanging, the launch reports SCC_ERR_TIMEOUT, and the context stays
usable (a later scc_run still gives the oracle's labels). The wait is made to
run out by a block that never arrives; nothing faults or hangs the GPU."""
import numpy as np
import pytest

import oracle
from paper_2303_04934_gb300 import graphgen as gg
from paper_2303_04934_gb300 import scc

from gpu_util import ensure_lib, labels_of, make_graph

pytestmark = pytest.mark.gpu


def test_grid_barrier_passes_when_every_block_arrives():
    ensure_lib()
    rc, arrived = scc.scc_debug_barrier_timeout(-1, 10**8)
    assert rc == scc.SCC_OK
    assert arrived >= 1


def test_grid_barrier_wait_runs_out_and_the_context_stays_usable():
    ensure_lib()
    for absent in (0, 3):
        rc, arrived = scc.scc_debug_barrier_timeout(absent, 10**6)  # 1 ms limit
        assert rc == scc.SCC_ERR_TIMEOUT, absent
        assert arrived == 0, absent
    g = gg.torus(2, 64, 0.5, seed=81)
    with make_graph(g) as G:
        assert np.array_equal(labels_of(G), oracle.scc_labels(g.n, g.offsets, g.targets)[0])
    rc, arrived = scc.scc_debug_barrier_timeout(-1, 10**8)
    assert rc == scc.SCC_OK and arrived >= 1
