"""The synthetic inputs follow their stated recipes: R-MAT without self-loops or
duplicate arcs and with ids permuted, tori whose arcs join lattice neighbours
with the stated density, exact k-NN graphs, and every generator independent of
the number of host threads. CPU only."""
import numpy as np
import pytest

from paper_2303_04934_gb300 import graphgen as gg


def _same(a, b):
    return a.n == b.n and np.array_equal(a.offsets, b.offsets) and np.array_equal(a.targets, b.targets)


def _arc_keys(g):
    e = gg.edges_of(g)
    return e[:, 0] * g.n + e[:, 1]


def test_rmat_recipe():
    scale, ef = 14, 16
    g = gg.rmat(scale, ef, seed=0x5CC01)
    n = 1 << scale
    assert g.n == n and len(g.offsets) == n + 1 and g.offsets[0] == 0
    assert np.all(np.diff(g.offsets) >= 0) and g.m == len(g.targets)
    assert g.targets.min() >= 0 and g.targets.max() < n
    e = gg.edges_of(g)
    assert not np.any(e[:, 0] == e[:, 1]), "self-loops are removed"
    keys = _arc_keys(g)
    assert len(np.unique(keys)) == g.m, "duplicate arcs are removed"
    # 2^18 samples, of which duplicates and self-loops are dropped: a skewed
    # quadrant distribution repeats many arcs, but most survive
    assert 0.6 * ef * n < g.m <= ef * n
    indeg = np.bincount(g.targets, minlength=n)
    outdeg = np.diff(g.offsets)
    assert indeg.max() > 20 * indeg.mean() and outdeg.max() > 20 * outdeg.mean()
    # ids are permuted: without it vertex 0 (the a-quadrant corner) has the most arcs
    unperm = gg.rmat(scale, ef, seed=0x5CC01, permute=False)
    assert np.argmax(np.diff(unperm.offsets)) == 0
    assert np.argmax(outdeg) != 0
    assert unperm.m == g.m and sorted(np.diff(unperm.offsets)) == sorted(outdeg)


def test_rmat_is_seeded_and_thread_independent():
    a = gg.rmat(12, 8, seed=5, threads=1)
    assert _same(a, gg.rmat(12, 8, seed=5, threads=4))
    assert _same(a, gg.rmat(12, 8, seed=5))
    assert not _same(a, gg.rmat(12, 8, seed=6))


@pytest.mark.parametrize("dims,side,p", [(2, 64, 0.5), (3, 20, 0.3), (2, (40, 25), 0.75)])
def test_torus_recipe(dims, side, p):
    g = gg.torus(dims, side, p, seed=0x5CC02)
    sides = (side,) * dims if isinstance(side, int) else side
    sides = list(sides) + [1] * (3 - len(sides))
    X, Y, Z = sides
    n = X * Y * Z
    assert g.n == n
    e = gg.edges_of(g)
    u, v = e[:, 0], e[:, 1]
    cu = np.stack([u % X, (u // X) % Y, u // (X * Y)], 1)
    cv = np.stack([v % X, (v // X) % Y, v // (X * Y)], 1)
    d = (cv - cu) % np.array(sides)
    step = (d == 1) | (d == np.array(sides) - 1)  # one step forward or back on the ring
    moved = d != 0
    assert np.all(moved.sum(1) == 1), "each arc changes one coordinate"
    assert np.all(step[moved]), "... by one step on its ring"
    assert len(np.unique(_arc_keys(g))) == g.m or min(sides[:dims]) <= 2
    # each of the 2*dims arcs of a vertex is present with probability p
    trials = 2 * dims * n
    sd = np.sqrt(trials * p * (1 - p))
    assert abs(g.m - trials * p) < 5 * sd
    assert _same(g, gg.torus(dims, side, p, seed=0x5CC02, threads=1))
    assert _same(g, gg.torus(dims, side, p, seed=0x5CC02, threads=3))


def test_knn_is_exact():
    n, k = 3000, 5
    g, pts = gg.knn(n, k, seed=0x5CC03, return_points=True)
    assert g.n == n and g.m == n * k and np.all(np.diff(g.offsets) == k)
    assert pts.shape == (n, 3) and pts.dtype == np.float32
    diff = pts[:, None, :].astype(np.float64) - pts[None, :, :].astype(np.float64)
    d2 = (diff * diff).sum(-1)
    np.fill_diagonal(d2, np.inf)  # itself excluded
    nbrs = g.targets.reshape(n, k)
    assert not np.any(nbrs == np.arange(n)[:, None])
    assert all(len(set(r)) == k for r in nbrs.tolist())
    chosen = np.take_along_axis(d2, nbrs, 1)
    others = d2.copy()
    np.put_along_axis(others, nbrs, np.inf, 1)
    # the chosen k are the k nearest: the farthest chosen is no farther than the
    # nearest left out (up to float32 rounding of the generator's distances)
    far, near = chosen.max(1), others.min(1)
    assert np.all(far <= near * (1 + 1e-5) + 1e-12)


def test_knn_is_seeded_and_thread_independent():
    a = gg.knn(20000, 4, seed=9, threads=1)
    assert _same(a, gg.knn(20000, 4, seed=9, threads=4))
    assert not _same(a, gg.knn(20000, 4, seed=10))
