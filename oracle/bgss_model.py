"""A sequential model of the BGSS method (Alg. 1) with this library's readings
of the paper -- TEST INFRASTRUCTURE ONLY (see the package docstring).

It takes the method's steps in the paper's order on small graphs, with plain
Python sets and breadth-first searches, so that a reader can check each step
against the paper; the tests compare its labels with Tarjan's. It shows that the
readings the CUDA path implements reach the exact SCC partition:

* trimming once at the start, self-loops not counted (Sec. 4.1);
* the seeded pivot order over the untrimmed vertices, batch 0 = the first pivot
  alone, batch sizes ceil(beta^i) (Alg. 1; Sec. 4.3);
* the first SCC by one forward and one backward single-reachability search from
  the first pivot (Sec. 4.2); the vertices it leaves form three classes;
* trimming inside a class: a vertex with no arc from, or no arc to, an
  unfinished vertex of its own class is a singleton SCC, in passes;
* per batch, forward and backward reachability from every source, following an
  arc only when both ends are unfinished and in the source's class (Alg. 1;
  Sec. 4.3-4.4); a vertex reached both ways from a source s is in s's SCC and is
  labelled by the largest such source (Sec. 4.4); every other reached vertex
  moves to the class (old class, largest forward source, largest backward
  source);
* the output label of a vertex is the smallest vertex id of its SCC;
* optionally, the batched kernel's cut of the order (the library's reading
  r17): further batches of one pivot after the first while a step leaves at
  least 1/8 of the active vertices reached one way only, the batches of Alg. 1
  after the positions those steps took, and a batch of at most
  ``single_fallback`` sources whose pairs in one direction exceed ``pair_cap``
  taken one pivot at a time (on the GPU: a batch whose pair tables overflow).
"""
from __future__ import annotations

from collections import deque

import numpy as np

from . import batch_bounds, pivot_order

NONE = -1


def _reach(adj, s, cls, done):
    """Vertices reached from s along arcs whose ends are unfinished and in s's class."""
    c = cls[s]
    seen = {s}
    q = deque([s])
    while q:
        u = q.popleft()
        for v in adj[u]:
            if v not in seen and not done[v] and cls[v] == c:
                seen.add(v)
                q.append(v)
    return seen


def _single_step(out, inn, p, cls, done, rep):
    """One single-pivot step inside p's class: reached both ways -> p's SCC,
    one way -> class (old class, p or none, p or none). Returns (finished,
    reached one way only)."""
    f = _reach(out, p, cls, done)
    b = _reach(inn, p, cls, done)
    fin = one = 0
    for v in f | b:
        if v in f and v in b:
            done[v] = True
            rep[v] = p
            fin += 1
        else:
            cls[v] = (cls[v], p if v in f else NONE, p if v in b else NONE)
            one += 1
    return fin, one


def bgss_labels(n: int, offsets, targets, beta: float = 2.0, seed: int = 0x5CC00, class_trim: bool = True,
                single_steps: int = 0, single_fallback: int = 0, pair_cap: int = 0):
    """SCC labels (smallest vertex id of each SCC) by the model of Alg. 1.

    ``single_steps`` > 0 selects the batched kernel's cut of the pivot order
    (at most that many single-pivot steps in all before the batches), with
    ``single_fallback`` / ``pair_cap`` its per-source fallback for small
    batches; 0 keeps the paper's cut. Returns (labels, stats) with stats =
    dict(n_trimmed, first_scc_size, n_class_trimmed, batches, single_steps,
    fallback_batches)."""
    off = np.asarray(offsets, dtype=np.int64)
    tg = np.asarray(targets, dtype=np.int64)
    out = [[] for _ in range(n)]
    inn = [[] for _ in range(n)]
    for u in range(n):
        for v in tg[off[u]:off[u + 1]].tolist():
            if v != u:  # self-loops never change an SCC
                out[u].append(v)
                inn[v].append(u)
    rep = list(range(n))       # SCC representative of finished vertices
    done = [False] * n
    cls = [0] * n              # class of unfinished vertices (a tuple after the first split)
    stats = dict(n_trimmed=0, first_scc_size=0, n_class_trimmed=0, batches=0, single_steps=0, fallback_batches=0)

    # trimming once (Sec. 4.1)
    for v in range(n):
        if not out[v] or not inn[v]:
            done[v] = True
            stats["n_trimmed"] += 1
    active = np.array([0 if done[v] else 1 for v in range(n)], np.uint8)
    order = pivot_order(active, seed).tolist()
    bounds = batch_bounds(len(order), beta).tolist()

    # the first SCC from the first pivot (Sec. 4.2)
    if order:
        s0 = order[0]
        f = _reach(out, s0, cls, done)
        b = _reach(inn, s0, cls, done)
        for v in f & b:
            done[v] = True
            rep[v] = s0
        stats["first_scc_size"] = len(f & b)
        for v in range(n):
            if not done[v]:
                cls[v] = (cls[v], s0 if v in f else NONE, s0 if v in b else NONE)
        stats["batches"] = 1
        stats["single_steps"] = 1
        pos = 1  # pivot positions taken
        if single_steps > 0:
            # further steps while the last one left at least 1/8 of the active
            # vertices reached one way only (the first step's count included)
            active_before = len(order)
            one = len((f | b) - (f & b))
            while stats["single_steps"] < single_steps and 8 * one >= active_before and pos < len(order):
                while pos < len(order) and done[order[pos]]:
                    pos += 1
                if pos == len(order):
                    break
                active_before = sum(1 for v in range(n) if not done[v])
                _, one = _single_step(out, inn, order[pos], cls, done, rep)
                pos += 1
                stats["single_steps"] += 1

        # trimming inside the classes, in passes while one still finishes a vertex
        while class_trim:
            fin = [v for v in range(n) if not done[v] and (
                not any(not done[u] and cls[u] == cls[v] for u in inn[v]) or
                not any(not done[w] and cls[w] == cls[v] for w in out[v]))]
            for v in fin:
                done[v] = True
            stats["n_class_trimmed"] += len(fin)
            if not fin:
                break

    # prefix-doubling batches (Alg. 1; Sec. 4.3-4.4); batch 0 was the first SCC.
    # The batched kernel's cut starts after the single-pivot steps' positions
    # with widths beta, beta^2, ... (ceil of each)
    if single_steps > 0 and order:
        cut = [pos]
        width = beta
        while cut[-1] < len(order):
            cut.append(min(len(order), cut[-1] + int(np.ceil(width))))
            width *= beta
        ranges = list(zip(cut[:-1], cut[1:]))
    else:
        ranges = [(bounds[i], bounds[i + 1]) for i in range(1, len(bounds) - 1)]
    for lo, hi in ranges:
        srcs = [s for s in order[lo:hi] if not done[s]]
        if not srcs:
            continue
        stats["batches"] += 1
        fmax = [NONE] * n
        bmax = [NONE] * n
        hit = [NONE] * n
        fwd = {s: _reach(out, s, cls, done) for s in srcs}
        bwd = {s: _reach(inn, s, cls, done) for s in srcs}
        if (single_fallback and len(srcs) <= single_fallback and
                max(sum(len(x) for x in fwd.values()), sum(len(x) for x in bwd.values())) > pair_cap):
            # the batch's pairs overflow: one single-pivot step per source, in order
            stats["fallback_batches"] += 1
            for s_ in srcs:
                if not done[s_]:
                    _single_step(out, inn, s_, cls, done, rep)
                    stats["single_steps"] += 1
            continue
        for s in srcs:
            for v in fwd[s]:
                fmax[v] = max(fmax[v], s)
                if v in bwd[s]:
                    hit[v] = max(hit[v], s)
            for v in bwd[s]:
                bmax[v] = max(bmax[v], s)
        for v in range(n):
            if done[v]:
                continue
            if hit[v] != NONE:
                done[v] = True
                rep[v] = hit[v]
            elif fmax[v] != NONE or bmax[v] != NONE:
                cls[v] = (cls[v], fmax[v], bmax[v])
    assert all(done), "every vertex is finished once every pivot has been a source"

    # canonical labels: the smallest vertex of each SCC
    low = {}
    for v in range(n):
        low[rep[v]] = min(low.get(rep[v], v), v)
    return np.array([low[rep[v]] for v in range(n)], np.int32), stats
