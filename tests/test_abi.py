"""The C-ABI library builds and exports every entry point include/dmwf.h declares
(no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:dm_status|void|const char \*)\s*\*?\s*(dm_\w+)\s*\(", src, re.M))
    return names


@pytest.fixture(scope="module")
def built_lib():
    from paper_1801_05358_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["dm_plan_create", "dm_set_spectra", "dm_set_noise_mask", "dm_wiener_filter",
              "dm_constrained_realization"]:
        assert n in names


def test_library_exports_every_declared_symbol(built_lib):
    missing = [n for n in sorted(_declared()) if not hasattr(built_lib, n)]
    assert not missing, missing


def test_binding_lists_match_header():
    from paper_1801_05358_gb300 import dmwf
    assert set(dmwf.EXPORTS) <= _declared()


def test_binding_fails_loudly_without_library(monkeypatch):
    from paper_1801_05358_gb300 import dmwf
    monkeypatch.setattr(dmwf, "_lib", None)
    monkeypatch.setattr(dmwf, "LIB_PATH", "/nonexistent/libdmwf.so")
    with pytest.raises(ImportError):
        dmwf.lib()
