"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
symbol that include/*.h declares; host-side argument checks. CPU only."""
import ctypes
import os
import re

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


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    monkeypatch.setattr(scc, "_lib", None)
    monkeypatch.setattr(libbuild, "SO_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        scc.load()
