"""The C ABI library builds, loads without a GPU, and exports every symbol
include/gko.h declares; the binding covers the header; the product package
never reaches the oracle."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_2006_14290_gb300 import build as B
from paper_2006_14290_gb300 import gko as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared():
    names = []
    for h in HEADERS:
        with open(h) as f:
            names += re.findall(r"^GKO_API [^(;]*?\b(gko_\w+)\(", f.read(), re.M)
    return names


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    return B.build()


def test_header_declares_the_boundary():
    names = declared()
    for need in ("gko_matrix_create_csr", "gko_matrix_convert_to_ell", "gko_matrix_convert_to_coo",
                 "gko_matrix_convert_to_hybrid", "gko_spmv", "gko_dot", "gko_spmv_dot"):
        assert need in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared() if not hasattr(L, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\s(gko_\w+)$", out, re.M))
    assert set(declared()) <= exported


def test_binding_matches_header():
    names = set(declared())
    bound = set(G.SIGNATURES) | set(G.OPTIONAL)
    assert names <= bound, names - bound
    assert set(G.SIGNATURES) <= names


def test_struct_layouts_match_the_binding(tmp_path):
    """The ctypes mirrors of the header's structs have the C compiler's size
    and field offsets (a renamed, reordered or retyped field would otherwise
    pass garbage through the ABI)."""
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    structs = {"gko_solve_opts": G.SolveOpts, "gko_solve_result": G.SolveResult}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gko.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    r = subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True).stdout
    got = dict(line.split() for line in out.splitlines() if line)
    assert len(got) == sum(1 + len(py._fields_) for py in structs.values())
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(py, fname).offset, (cname, fname)


def test_host_only_calls_work_without_gpu(libpath):
    L = ctypes.CDLL(libpath)
    L.gko_status_string.restype = ctypes.c_char_p
    assert L.gko_status_string(4) == b"not converged"
    assert L.gko_version() >= 100
    assert L.gko_set_memory_budget(ctypes.c_int64(-1)) == 1  # INVALID_ARG
    assert L.gko_set_memory_budget(ctypes.c_int64(0)) == 0


def test_product_package_does_not_reach_the_oracle():
    pkg = os.path.join(ROOT, "paper_2006_14290_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                with open(os.path.join(dirpath, f)) as fh:
                    src = fh.read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), f
                assert "gko_oracle" not in src and "liboracle" not in src, f
