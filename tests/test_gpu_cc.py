"""GPU connected components (cc_run: LDD-UF-JTB with VGC and the hash bag,
Sec. 5.1, Alg. 4) are bit-identical to the CPU oracle (union-find on the
undirected graph under the arcs, label = smallest vertex id of the component)
on edge cases, small random graphs, lattices with many components, R-MAT and
k-NN graphs, for host and device buffers and on repeated calls (the symmetric
CSR kept with the handle). The labels are canonical, so the decomposition's
races (which centre claims a vertex) cannot change them."""
import numpy as np
import pytest

import oracle
from paper_2303_04934_gb300 import graphgen as gg
from paper_2303_04934_gb300 import scc

from gpu_util import ensure_lib, make_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _cc(G, host=False):
    import torch
    if host:
        out = np.empty(G.n, np.int32)
        scc.cc_run(G.h, out)
        return out
    out = torch.empty(max(G.n, 1), dtype=torch.int32, device="cuda")
    scc.cc_run(G.h, out[:G.n] if G.n else out)
    torch.cuda.synchronize()
    return out.cpu().numpy()[:G.n]


def _check(g, host=False, reps=1):
    want, ncc = oracle.cc_labels(g.n, g.offsets, g.targets)
    with make_graph(g, on_device=not host) as G:
        for _ in range(reps):
            got = _cc(G, host=host)
            assert np.array_equal(got, want), g.name
        st = scc.cc_get_stats(G.h)
    if g.n:
        assert st["components"] == ncc, g.name
        assert ncc <= st["clusters"] <= g.n, g.name
    return st


def test_edge_cases():
    _check(gg.from_edges(0, [], name="empty"))
    _check(gg.from_edges(1, [], name="one"))
    _check(gg.from_edges(1, [(0, 0)], name="one_self_loop"))
    _check(gg.from_edges(6, [], name="no_arcs"))
    _check(gg.from_edges(4, [(i, i) for i in range(4)], name="self_loops_only"))
    _check(gg.from_edges(5, [(4, 3), (3, 2), (2, 1), (1, 0)], name="path_backwards"))
    _check(gg.from_edges(6, [(0, 1), (0, 1), (1, 0), (5, 4)], name="duplicates"))
    _check(gg.from_edges(7, [(6, 0), (1, 2), (3, 4), (4, 5), (5, 3)], name="mixed"))


def test_small_random_graphs():
    rng = np.random.default_rng(0xCC5)
    for i in range(60):
        n = int(rng.integers(2, 400))
        p = float(rng.choice([0.001, 0.005, 0.01, 0.05]))
        _check(gg.gnp(n, p, seed=900 + i, allow_self=bool(i % 2)))


@pytest.mark.parametrize("make", [
    lambda: gg.torus(2, 256, 0.5, seed=0x5CC00),
    lambda: gg.torus(2, 300, 0.15, seed=31),
    lambda: gg.torus(3, 40, 0.1, seed=32),
    lambda: gg.rmat(16, 8, seed=33),
    lambda: gg.rmat(18, 2, seed=34),
    lambda: gg.knn(200_000, 3, seed=35),
    lambda: gg.paper_lattice(300, 300, 1, seed=36),
], ids=["torus2d_256", "torus2d_sparse", "torus3d_sparse", "rmat16", "rmat18_ef2", "knn200k", "rec_prime_300"])
def test_medium_graphs_device_and_host(make):
    g = make()
    _check(g, host=False, reps=2)
    _check(g, host=True)


def test_component_labels_refined_by_scc_labels():
    """Every SCC lies inside one component: cc[scc_label[v]] == cc[v] on the GPU's outputs."""
    g = gg.rmat(15, 4, seed=41)
    with make_graph(g) as G:
        import torch
        lab = torch.empty(g.n, dtype=torch.int32, device="cuda")
        scc.scc_run(G.h, lab)
        cc = _cc(G)
        lab = lab.cpu().numpy()
    assert np.array_equal(cc[lab], cc)


@pytest.mark.parametrize("ldd_beta", [1.2, 2.0, 8.0])
def test_labels_do_not_depend_on_the_batch_growth(ldd_beta):
    """The decomposition's batch growth (the paper's 1.2, the default 2, a
    coarse 8) changes the clusters, never the components."""
    c = scc.scc_config_default()
    c.ldd_beta = ldd_beta
    for g in (gg.rmat(15, 8, seed=51), gg.torus(2, 120, 0.3, seed=52), gg.knn(50_000, 4, seed=53)):
        want, ncc = oracle.cc_labels(g.n, g.offsets, g.targets)
        with make_graph(g, config=c) as G:
            got = _cc(G)
            st = scc.cc_get_stats(G.h)
        assert np.array_equal(got, want), (g.name, ldd_beta)
        assert st["components"] == ncc
