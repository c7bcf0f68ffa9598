"""Properties every correct SCC labelling has -- test infrastructure only.

For a labelling ``lab`` with ``lab[v]`` = the smallest vertex id of v's SCC
(Sec. 1 problem statement with the canonical minimum):

1. canonical minimum: ``lab[v] <= v`` and ``lab[lab[v]] == lab[v]``;
2. closed classes: every arc (u, v) whose endpoints share a label lies in a
   directed cycle of that class, i.e. the class is strongly connected -- checked
   by a forward and a backward search from the class's minimum restricted to the
   class;
3. the condensation (arcs between different labels) is acyclic -- Kahn's
   algorithm removes every class.

Together these characterise the SCC partition: (2) says every class is strongly
connected, (3) says no two classes can be merged.
"""
from __future__ import annotations

import numpy as np


def check_scc_labels(n: int, offsets, targets, lab) -> None:
    lab = np.asarray(lab, dtype=np.int64)
    off = np.asarray(offsets, dtype=np.int64)
    adj = np.asarray(targets, dtype=np.int64)
    assert lab.shape == (n,)
    if n == 0:
        return
    v = np.arange(n)
    assert np.all(lab >= 0) and np.all(lab <= v), "label must be a vertex id <= v"
    assert np.all(lab[lab] == lab), "label must be a fixed point (canonical minimum)"
    src = np.repeat(v, np.diff(off))
    same = lab[src] == lab[adj]

    # (2) each class strongly connected: BFS from the class representative inside
    # the class on G and on G^T reaches the whole class.
    for direction in (0, 1):
        a, b = (src, adj) if direction == 0 else (adj, src)
        a, b = a[same], b[same]
        order = np.argsort(a, kind="stable")
        a, b = a[order], b[order]
        row = np.zeros(n + 1, np.int64)
        np.add.at(row, a + 1, 1)
        row = np.cumsum(row)
        seen = np.zeros(n, bool)
        frontier = np.unique(lab)
        seen[frontier] = True
        while len(frontier):
            starts, ends = row[frontier], row[frontier + 1]
            cnt = ends - starts
            if cnt.sum() == 0:
                break
            idx = np.repeat(starts - np.concatenate([[0], np.cumsum(cnt)[:-1]]), cnt) + np.arange(cnt.sum())
            nb = b[idx]
            nb = np.unique(nb[~seen[nb]])
            seen[nb] = True
            frontier = nb
        assert seen.all(), "a label class is not strongly connected"

    # (3) condensation acyclic (Kahn).
    cu, cv = lab[src[~same]], lab[adj[~same]]
    if len(cu):
        pairs = np.unique(cu * n + cv)
        cu, cv = pairs // n, pairs % n
    classes = np.unique(lab)
    indeg = np.zeros(n, np.int64)
    np.add.at(indeg, cv, 1)
    order = np.argsort(cu, kind="stable")
    cu, cv = cu[order], cv[order]
    row = np.zeros(n + 1, np.int64)
    np.add.at(row, cu + 1, 1)
    row = np.cumsum(row)
    ready = [int(c) for c in classes if indeg[c] == 0]
    removed = 0
    while ready:
        c = ready.pop()
        removed += 1
        for d in cv[row[c]:row[c + 1]]:
            indeg[d] -= 1
            if indeg[d] == 0:
                ready.append(int(d))
    assert removed == len(classes), "the condensation has a cycle"
