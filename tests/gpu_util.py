"""Helpers for the GPU parity tests (imported only by tests marked gpu)."""
from __future__ import annotations

import numpy as np

from paper_2303_04934_gb300 import build as libbuild
from paper_2303_04934_gb300 import scc


def ensure_lib():
    libbuild.build()
    return scc.load()


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make_graph(g, config=None, on_device=True):
    """SccGraph of a graphgen.Graph, input copied from device (or host) memory."""
    if on_device:
        return scc.SccGraph(g.n, dev(g.offsets), dev(g.targets), config=config)
    return scc.SccGraph(g.n, np.ascontiguousarray(g.offsets), np.ascontiguousarray(g.targets), config=config)


def config(**kw):
    c = scc.scc_config_default()
    for k, v in kw.items():
        setattr(c, "lambda_" if k == "lam" else k, v)
    return c


def labels_of(G, host=False):
    import torch
    if host:
        out = np.empty(G.n, np.int32)
        scc.scc_run(G.h, out)
        return out
    out = torch.empty(max(G.n, 1), dtype=torch.int32, device="cuda")
    scc.scc_run(G.h, out[:G.n] if G.n else out)
    torch.cuda.synchronize()
    return out.cpu().numpy()[:G.n]


def self_loop_free(g):
    """Forward CSR with self-loops removed, row order kept (the library's G)."""
    src = np.repeat(np.arange(g.n), np.diff(g.offsets.astype(np.int64)))
    keep = src != g.targets
    cnt = np.bincount(src[keep], minlength=g.n)
    off = np.zeros(g.n + 1, np.int32)
    off[1:] = np.cumsum(cnt)
    return off, g.targets[keep].astype(np.int32)


def sorted_rows(off, adj):
    """adj with every CSR row sorted increasingly."""
    off = np.asarray(off, dtype=np.int64)
    row = np.repeat(np.arange(len(off) - 1), np.diff(off))
    order = np.lexsort((adj, row))
    return np.asarray(adj)[order]
