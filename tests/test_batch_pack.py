"""Packed batches (host side of include/scc_batch.h): packing keeps every graph
intact and the mixed generator follows its size and family recipe."""
import numpy as np

from paper_2303_04934_gb300 import graphgen as gg


def test_pack_roundtrip():
    gs = [gg.from_edges(0, []), gg.gnp(30, 0.1, seed=1, allow_self=True), gg.torus(2, 5, 0.5, seed=2),
          gg.from_edges(3, [(0, 1), (1, 0), (2, 2)])]
    p = gg.pack(gs)
    assert p.G == 4 and p.vbase.tolist() == [0, 0, 30, 55, 58]
    assert len(p.offsets) == p.vbase[-1] + p.G and len(p.targets) == p.ebase[-1]
    for i, g in enumerate(gs):
        h = p.graph(i)
        assert h.n == g.n and np.array_equal(h.offsets, g.offsets) and np.array_equal(h.targets, g.targets)
    lab = np.arange(p.vbase[-1])
    assert p.labels_of(lab, 2).tolist() == list(range(30, 55))


def test_mixed_spec_recipe():
    spec = gg.mixed_batch_spec(400, 1000, 1_000_000, seed=9)
    kinds = [k for k, _, _ in spec]
    assert kinds[::2] == ["torus"] * 200 and kinds[1::2] == ["rmat"] * 200
    sides = np.array([s for k, s, _ in spec if k == "torus"])
    scales = np.array([s for k, s, _ in spec if k == "rmat"])
    assert sides.min() >= 31 and sides.max() <= 1000
    assert scales.min() >= 10 and scales.max() <= 20
    # log-uniform: about half of the sizes below the geometric mean (31.6k)
    n_t = sides.astype(float) ** 2
    assert 0.35 < np.mean(n_t < 31623) < 0.65
    assert gg.mixed_batch_spec(400, 1000, 1_000_000, seed=9) == spec
