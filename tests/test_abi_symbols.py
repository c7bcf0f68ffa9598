"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
symbol that include/*.h declares; host-side argument checks. CPU only."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2303_04934_gb300 import build as libbuild
from paper_2303_04934_gb300 import scc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^SCC_API\s+[\w\s\*]*?\b(\w+)\s*\(", text, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return scc.load()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert len(declared) >= 16
    assert sorted(declared) == sorted(scc.EXPORTED)
    for name in declared:
        assert hasattr(lib, name), name


def test_error_strings_and_default_config(lib):
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert lib.scc_error_string(code)
    cfg = scc.scc_config_default()
    assert cfg.tau == 0 and cfg.beta == 2.0 and cfg.sigma == 50 and cfg.lambda_ == 16384


def test_invalid_arguments_rejected_on_the_host(lib):
    h = ctypes.c_void_p()
    # negative n, m out of range, missing pointers: refused before any CUDA call
    assert lib.scc_graph_create(-1, 0, None, None, None, ctypes.byref(h)) == scc.SCC_ERR_INVALID_ARG
    assert lib.scc_graph_create(4, 2**31, None, None, None, ctypes.byref(h)) == scc.SCC_ERR_INVALID_ARG
    assert lib.scc_graph_create(4, 3, None, None, None, ctypes.byref(h)) == scc.SCC_ERR_INVALID_ARG
    assert lib.scc_run(None, None, None) == scc.SCC_ERR_INVALID_ARG
    assert lib.reach_multi(None, None, 1, 0, None, None) == scc.SCC_ERR_INVALID_ARG
    assert lib.scc_set_config(None, None) == scc.SCC_ERR_INVALID_ARG


def test_null_handles_and_bad_arguments_rejected_on_the_host(lib):
    """Every entry point that takes a handle refuses NULL (destroy calls accept
    it), and bad sizes are refused, before any CUDA call."""
    E = scc.SCC_ERR_INVALID_ARG
    i32, i64, dbl = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_double()
    for name, args in [
        ("scc_get_stats", (None, None)), ("scc_graph_info", (None, None, None, None)),
        ("cc_run", (None, None, None)), ("cc_get_stats", (None, None)),
        ("le_lists_run", (None, None, None)), ("le_lists_get", (None, None, None, None, None, None)),
        ("le_get_stats", (None, None)), ("scc_debug_le_lists", (None, 1, 1, None, None)),
        ("reach_multi_noalloc", (None, None, 1, 0, None, None)),
        ("scc_debug_csr", (None, 0, None, None, None)), ("scc_debug_trim", (None, None, None)),
        ("scc_debug_pivot_order", (None, None, ctypes.byref(i32), None)),
        ("scc_debug_single_reach", (None, None, 0, 0, None, None)),
        ("scc_debug_multi_reach", (None, None, None, 1, 0, None, 0, ctypes.byref(i64), 0, None)),
        ("scc_debug_reach_multi_wide", (None, None, 1, 0, None, None)),
        ("scc_debug_barrier_timeout", (-1, 0, ctypes.byref(i32), None)),
        ("scc_debug_barrier_timeout", (-1, 10**6, None, None)),
        ("scc_debug_barrier_timeout", (-2, 10**6, ctypes.byref(i32), None)),
        ("scc_batch_create", (-1, None, None, None, None, None, None)),
        ("scc_batch_set_config", (None, None)), ("scc_batch_get_config", (None, None)),
        ("scc_batch_run", (None, None, None)), ("scc_batch_autotune", (None, 0, None, None, None)),
        ("scc_batch_get_stats", (None, None)), ("scc_debug_batch_times", (None, None)),
        ("scc_server_add_graph", (None, 1, 0, None, None, ctypes.byref(i32))),
        ("scc_server_remove_graph", (None, 0)),
        ("scc_server_submit_scc", (None, 1, 0, None, None, None, ctypes.byref(i64))),
        ("scc_server_submit_reach", (None, 0, None, 1, 0, None, ctypes.byref(i64))),
        ("scc_server_wait", (None, 1, ctypes.byref(i32), ctypes.byref(dbl))),
        ("scc_server_drain", (None,)), ("scc_server_get_stats", (None, None)), ("scc_server_reset_stats", (None,)),
    ]:
        assert getattr(lib, name)(*args) == E, name
    for name in ("scc_graph_destroy", "scc_batch_destroy", "scc_server_destroy"):
        assert getattr(lib, name)(None) == scc.SCC_OK, name
    # a server configuration out of range is refused before the server starts
    cfg = scc.scc_server_config()
    assert lib.scc_server_config_default(ctypes.byref(cfg)) == scc.SCC_OK
    for field, bad in (("mem_cap_bytes", 0), ("batch_graphs", 0), ("batch_vertices", -1), ("max_bypass_ms", -1.0)):
        c = scc.scc_server_config.from_buffer_copy(cfg)
        setattr(c, field, bad)
        h = ctypes.c_void_p()
        assert lib.scc_server_create(ctypes.byref(c), ctypes.byref(h)) == E, field
        assert not h.value


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    monkeypatch.setattr(scc, "_lib", None)
    monkeypatch.setattr(libbuild, "SO_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        scc.load()


def test_binding_checks_element_types_and_lengths(lib):
    """The binding refuses arrays the C ABI would misread (wrong element type)
    or overrun (too short) before calling the library: the graph below would
    otherwise reach CUDA, which this host does not have (SCC_ERR_CUDA)."""
    import torch
    off = np.array([0, 1, 2, 3, 3], np.int32)
    adj = np.array([1, 2, 0], np.int32)
    for o, a, word in [(off, adj.astype(np.int64), "targets"), (off.astype(np.int64), adj, "offsets"),
                       (off[:4], adj, "offsets"), (off, adj[:2], "targets"), (off, None, "targets"),
                       (torch.from_numpy(off), torch.from_numpy(adj).to(torch.int64), "targets")]:
        with pytest.raises(scc.SccError, match=word) as e:
            scc.scc_graph_create(4, 3, o, a)
        assert e.value.code == scc.SCC_ERR_INVALID_ARG
    # well-typed arguments pass the checks and reach the library
    if torch.cuda.is_available():
        scc.scc_graph_destroy(scc.scc_graph_create(4, 3, off, adj))
    else:
        with pytest.raises(scc.SccError) as e:
            scc.scc_graph_create(4, 3, off, adj)
        assert e.value.code == scc.SCC_ERR_CUDA
    # accepted element types: int32 ids, 64-bit masks of either signedness, numpy or torch
    for a, types, count in [(np.zeros(5, np.int32), scc.I32, 5), (torch.zeros(5, dtype=torch.int32), scc.I32, 5),
                            (np.zeros(3, np.uint64), scc.W64, 3), (torch.zeros(3, dtype=torch.int64), scc.W64, 3),
                            (np.zeros(4, np.int64), scc.I64, 2), (None, scc.I32, 0)]:
        scc._arr(a, "x", types, count)
    for a, types, count in [(np.zeros(5, np.uint32), scc.I32, 5), (np.zeros(3, np.float64), scc.W64, 3),
                            (np.zeros(2, np.uint64), scc.W64, 3), (None, scc.I32, 1),
                            (torch.zeros(3, dtype=torch.int32), scc.W64, 3)]:
        with pytest.raises(scc.SccError):
            scc._arr(a, "x", types, count)
