"""The public headers compile as plain C (no CUDA headers), and every structure
the Python binding mirrors has the same size and field offsets as in C. CPU
only: a small C program built with the host compiler prints the layouts."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_2303_04934_gb300 import scc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = ["scc.h", "scc_batch.h", "scc_serve.h", "scc_debug.h"]
STRUCTS = [scc.scc_config, scc.scc_stats, scc.scc_cc_stats, scc.scc_le_stats, scc.scc_batch_config, scc.scc_batch_stats, scc.scc_server_config,
           scc.scc_server_stats]


def _c_name(field):
    # `lambda` is a Python keyword: the binding spells the field `lambda_`
    return field[:-1] if field.endswith("_") else field


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    d = tmp_path_factory.mktemp("abi")
    lines = ["#include <stddef.h>", "#include <stdio.h>"]
    lines += [f'#include "{os.path.join(ROOT, "include", h)}"' for h in HEADERS]
    lines.append("int main(void) {")
    for st in STRUCTS:
        name = st.__name__
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {_c_name(f)}));')
    lines.append("  return 0;\n}")
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        name, field, value = line.split()
        table[(name, field)] = int(value)
    return table


@pytest.mark.parametrize("st", STRUCTS, ids=lambda s: s.__name__)
def test_binding_structs_match_the_headers(c_layout, st):
    name = st.__name__
    assert c_layout[(name, "sizeof")] == ctypes.sizeof(st)
    for f, _ in st._fields_:
        assert c_layout[(name, f)] == getattr(st, f).offset, f"{name}.{f}"


def _header_fields(name):
    text = "".join(open(os.path.join(ROOT, "include", h)).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), text, flags=re.S).group(1)
    names = []
    for decl in body.split(";"):
        if decl.strip():  # "type a, b, c": the last word of each declarator
            names += [re.findall(r"\w+", d)[-1] for d in decl.split(",")]
    return names


@pytest.mark.parametrize("st", STRUCTS, ids=lambda s: s.__name__)
def test_binding_mirrors_every_header_field_in_order(st):
    assert [_c_name(f) for f, _ in st._fields_] == _header_fields(st.__name__)
