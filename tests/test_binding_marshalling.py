"""The Python binding only marshals arguments: against a stand-in for the C
library that records its calls, every wrapper passes the sizes and pointers the
C ABI expects for numpy arrays, CPU torch tensors and slices, and refuses a
mistyped or short array without calling the library. CPU only."""

import numpy as np
import pytest
import torch

from paper_2303_04934_gb300 import graphgen as gg
from paper_2303_04934_gb300 import scc


class _Lib:
    """Records calls; fills the out-parameters the wrappers read back. Handles
    stay NULL, so that a wrapper collected after the test (when the real library
    is back) has nothing to destroy."""

    def __init__(self):
        self.calls = []
        self.n = 0
        self.nv = 0

    def __getattr__(self, name):
        def call(*args):
            self.calls.append((name, args))
            if name == "scc_graph_info":
                args[1]._obj.value = self.n
            elif name == "scc_batch_get_stats":
                args[1]._obj.vertices = self.nv
            elif name == "scc_server_add_graph":
                args[-1]._obj.value = 7
            elif name == "scc_error_string":
                return b"stand-in"
            return 0
        return call

    def last(self, name):
        return [a for nm, a in self.calls if nm == name][-1]


@pytest.fixture()
def lib(monkeypatch):
    fake = _Lib()
    monkeypatch.setattr(scc, "load", lambda: fake)
    return fake


def _addr(a):
    return a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr()


def test_graph_calls_pass_sizes_and_pointers(lib):
    g = gg.rmat(9, 4, seed=3)
    lib.n = g.n
    for off, adj in [(g.offsets, g.targets), (torch.from_numpy(g.offsets), torch.from_numpy(g.targets))]:
        G = scc.SccGraph(g.n, off, adj)
        n, m, po, pt = lib.last("scc_graph_create")[:4]
        assert (n, m, po, pt) == (g.n, g.m, _addr(off), _addr(adj))
        lab = np.empty(g.n, np.int32)
        scc.scc_run(G.h, lab)
        assert lib.last("scc_run")[:2] == (G.h, lab.ctypes.data)
        src = np.array([3, 1, 4], np.int32)
        out = torch.empty(g.n, dtype=torch.int64)
        scc.reach_multi(G.h, src, 3, 1, out)
        assert lib.last("reach_multi")[:5] == (G.h, src.ctypes.data, 3, 1, out.data_ptr())
    # a slice starting inside a larger buffer passes its own address
    buf = torch.zeros(g.m + 3, dtype=torch.int32)
    scc.SccGraph(g.n, g.offsets, buf[3:])
    assert lib.last("scc_graph_create")[3] == buf[3:].data_ptr()


def test_mistyped_or_short_arrays_never_reach_the_library(lib):
    g = gg.rmat(8, 4, seed=4)
    lib.n = g.n
    h = scc.scc_graph_create(g.n, g.m, g.offsets, g.targets)
    before = len(lib.calls)
    bad_calls = [
        lambda: scc.scc_graph_create(g.n, g.m, g.offsets, g.targets.astype(np.int64)),
        lambda: scc.scc_graph_create(g.n, g.m, g.offsets[:-1], g.targets),
        lambda: scc.scc_run(h, np.empty(g.n - 1, np.int32)),
        lambda: scc.scc_run(h, np.empty(g.n, np.uint32)),
        lambda: scc.reach_multi(h, np.zeros(2, np.int32), 3, 0, np.empty(g.n, np.uint64)),
        lambda: scc.reach_multi(h, np.zeros(3, np.int32), 3, 0, np.empty(g.n, np.int32)),
        lambda: scc.scc_batch_create(2, np.zeros(2, np.int64), np.zeros(3, np.int64), g.offsets, g.targets),
        lambda: scc.scc_batch_create(1, np.zeros(2, np.int32), np.zeros(2, np.int64), g.offsets, g.targets),
    ]
    for f in bad_calls:
        with pytest.raises(scc.SccError) as e:
            f()
        assert e.value.code == scc.SCC_ERR_INVALID_ARG
    # scc_run and reach_multi ask for the graph's size first; nothing else was called
    assert {nm for nm, _ in lib.calls[before:]} <= {"scc_graph_info", "scc_error_string"}


def test_batch_and_server_calls(lib):
    gs = [gg.torus(2, 5, 0.5, seed=2), gg.rmat(6, 4, seed=3)]
    p = gg.pack(gs)
    lib.nv = int(p.vbase[-1])
    B = scc.SccBatch(p)
    G, pv, pe, po, pt = lib.last("scc_batch_create")[:5]
    assert (G, pv, pe, po, pt) == (p.G, p.vbase.ctypes.data, p.ebase.ctypes.data, p.offsets.ctypes.data,
                                   p.targets.ctypes.data)
    B.labels(torch.empty(lib.nv, dtype=torch.int32))
    with pytest.raises(scc.SccError):
        B.labels(torch.empty(lib.nv - 1, dtype=torch.int32))
    g = gs[1]
    with scc.SccServer() as srv:
        gid = srv.add_graph(g.n, g.offsets, g.targets)
        assert lib.last("scc_server_add_graph")[1:3] == (g.n, g.m)
        lab = np.empty(g.n, np.int32)
        srv.submit_scc(g.n, g.offsets, g.targets, lab)
        assert lib.last("scc_server_submit_scc")[1:3] == (g.n, g.m)
        out = np.empty(g.n, np.uint64)
        srv.submit_reach(gid, [5, 6], 1, out)
        a = lib.last("scc_server_submit_reach")
        assert (a[1], a[3], a[4], a[5]) == (gid, 2, 1, out.ctypes.data)
        # the output must hold one mask per vertex of the resident graph
        with pytest.raises(scc.SccError):
            srv.submit_reach(gid, [5], 0, np.empty(g.n - 1, np.uint64))
        with pytest.raises(scc.SccError):
            srv.submit_scc(g.n, g.offsets, g.targets, np.empty(g.n - 1, np.int32))
