"""The C-ABI library builds for sm_103a, loads, and exports every entry point declared in
include/mc.h (no compute calls: this runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "mc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mc_[a-z_]+)\s*\(", src)) - {"mc_alloc_fn", "mc_free_fn"})


@pytest.fixture(scope="module")
def libpath():
    from paper_2602_13198_gb300 import build
    return build.build()


def test_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (mc_\w+)", out))
    decl = declared()
    assert decl, "no declarations parsed"
    missing = [d for d in decl if d not in exported]
    assert not missing, missing


def test_loads_and_reports_errors_without_compute(libpath):
    from paper_2602_13198_gb300 import mc
    L = mc.lib()
    assert L.mc_version().decode().startswith("mcgb")
    # invalid parameters are rejected before any device work
    import ctypes as C
    p = mc.ModelParams()
    h = C.c_void_p()
    rc = L.mc_init_model(C.byref(h), C.byref(p))
    assert rc == -1 and h.value is None
    assert L.mc_last_error(None)


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2602_13198_gb300 import mc
    monkeypatch.setattr(mc, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(mc, "_lib", None)
    with pytest.raises(mc.MCError):
        mc.lib()
