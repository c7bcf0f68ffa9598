"""Oracle output checked against invariants (with planted mistakes that the
checker must catch) and against the paper's Table 2 statistics for its own
lattice models. CPU only."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle.invariants import check_scc_labels
from paper_2303_04934_gb300 import graphgen as gg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_scc_table_lattices.json")


@pytest.mark.parametrize("make", [
    lambda: gg.torus(2, 64, 0.5, seed=1),
    lambda: gg.torus(3, 16, 0.3, seed=2),
    lambda: gg.rmat(12, 8, seed=3),
    lambda: gg.knn(5000, 5, seed=4),
    lambda: gg.paper_lattice(60, 50, 0, seed=5),
    lambda: gg.paper_lattice(60, 50, 1, seed=6),
])
def test_tarjan_output_satisfies_invariants(make):
    g = make()
    lab, nscc = oracle.scc_labels(g.n, g.offsets, g.targets)
    check_scc_labels(g.n, g.offsets, g.targets, lab)
    assert nscc == len(np.unique(lab))


def test_checker_catches_planted_mistakes():
    g = gg.torus(2, 40, 0.5, seed=9)
    lab, _ = oracle.scc_labels(g.n, g.offsets, g.targets)
    sizes = np.bincount(lab, minlength=g.n)
    big = int(np.argmax(sizes))
    members = np.flatnonzero(lab == big)
    assert len(members) > 3
    # 1) split an SCC: one member gets its own label
    bad = lab.copy()
    bad[members[-1]] = members[-1]
    with pytest.raises(AssertionError):
        check_scc_labels(g.n, g.offsets, g.targets, bad)
    # 2) merge two SCCs that are not strongly connected
    other = int(np.flatnonzero((sizes == 1) & (np.arange(g.n) > big))[0])
    bad = lab.copy()
    bad[other] = big
    with pytest.raises(AssertionError):
        check_scc_labels(g.n, g.offsets, g.targets, bad)
    # 3) right partition, wrong representative (max instead of min)
    bad = lab.copy()
    bad[members] = members.max()
    with pytest.raises(AssertionError):
        check_scc_labels(g.n, g.offsets, g.targets, bad)
    # 4) merge a cycle of classes (condensation cycle) is caught
    e = [(0, 1), (1, 0), (2, 3), (3, 2), (1, 2)]
    gg_ = gg.from_edges(4, e)
    check_scc_labels(4, gg_.offsets, gg_.targets, np.array([0, 0, 2, 2]))
    with pytest.raises(AssertionError):
        check_scc_labels(4, gg_.offsets, gg_.targets, np.array([0, 0, 0, 0]))


@pytest.mark.slow
@pytest.mark.parametrize("name", ["REC", "REC'"])
def test_paper_table2_lattice_statistics(name):
    """Table 2 prints m, #SCC and |SCC1| for one random instance of each lattice
    model (Sec. 6 'Setup'); our generator + Tarjan draw another instance.

    REC' (independent arcs, p = 0.3 each way) is a pin: #SCC within 1% and the
    largest SCC of the same size (tens of vertices). REC (each vertex orients
    the arc to each neighbour at random, duplicates removed) reproduces m and
    |SCC1|/n within 0.2 percentage points but has ~10% fewer SCCs than the
    printed instance under every reading of the model text we found, so only a
    loose band is asserted there."""
    spec = json.load(open(GOLDEN))["graphs"][name]
    g = gg.paper_lattice(spec["X"], spec["Y"], spec["model"], seed=0x5CC00)
    assert g.n == spec["n"]
    assert abs(g.m - spec["m_paper"]) / spec["m_paper"] < 0.002
    lab, nscc = oracle.scc_labels(g.n, g.offsets, g.targets)
    scc1 = int(np.bincount(lab).max())
    if spec["model"] == 0:
        assert abs(nscc - spec["nscc_paper"]) / spec["nscc_paper"] < 0.15, nscc
        assert abs(scc1 - spec["scc1_paper"]) / g.n < 0.002, scc1
    else:
        assert abs(nscc - spec["nscc_paper"]) / spec["nscc_paper"] < 0.01, nscc
        assert 20 <= scc1 <= 100, scc1
