"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/spadj.h
declares; the binding fails loudly when the library is missing (no CPU fallback)."""
import ctypes
import os
import re

import pytest

from paper_2506_14792_gb300 import build, spadj

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "spadj.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(spadj_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    if build.stale():
        build.build()
    return build.LIB


def test_exports_every_declared_symbol(libpath):
    syms = declared_symbols()
    assert "spadj_gradient" in syms and "spadj_create" in syms
    L = ctypes.CDLL(libpath)
    missing = [s for s in syms if not hasattr(L, s)]
    assert not missing, missing


def test_binding_covers_header(libpath):
    assert set(declared_symbols()) <= set(spadj._SIGS)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(spadj, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(spadj, "_lib", None)
    with pytest.raises(RuntimeError):
        spadj.lib()


def test_create_rejects_bad_descriptor(libpath):
    d = spadj.spadj_desc()
    d.eq, d.scheme, d.batch, d.dt = 0, 2, 0, 1e-3
    h = ctypes.c_void_p()
    st = spadj.lib().spadj_create(ctypes.byref(d), None, ctypes.byref(h))
    assert st == spadj.SPADJ_ERR_INVALID
    assert b"batch" in spadj.lib().spadj_last_error(None)
