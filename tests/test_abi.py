"""The C-ABI library loads without a GPU and exports every entry point that
include/bf.h declares (no compute calls here)."""
import os
import re
import subprocess

import pytest

from paper_2512_12151_b300 import binding as B
from paper_2512_12151_b300 import build as build_mod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    hdr = open(os.path.join(ROOT, "include", "bf.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(bf_[a-z_0-9]+)\s*\(", hdr)))


@pytest.fixture(scope="module")
def libpath():
    return build_mod.build()


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    names = declared()
    assert len(names) >= 25
    missing = [n for n in names if n not in syms]
    assert not missing, missing


def test_binding_loads_and_covers_header(libpath):
    L = B.lib()
    for n in declared():
        assert hasattr(L, n)
        assert hasattr(B, n), f"binding lacks {n}"
    assert B.bf_status_str(0) == "ok"
    assert B.bf_status_str(-9) == "work buffer capacity exceeded"


def test_binding_fails_loudly_without_library(monkeypatch):
    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "LIB_PATH", "/nonexistent/libbf.so")
    with pytest.raises(RuntimeError, match="not built"):
        B.lib()


def test_struct_layouts_match_header():
    import ctypes as C
    # bf_params: 13 doubles + 7 int32 (padded to 8 bytes); bf_step_stats: 8 int32 + 6 doubles
    assert C.sizeof(B.bf_params) == 13 * 8 + 8 * 4
    assert C.sizeof(B.bf_step_stats) == 8 * 4 + 6 * 8
    assert C.sizeof(B.bf_mesh_desc) == 4 * 4 + 8 * 8
