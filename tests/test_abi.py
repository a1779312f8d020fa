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


def test_binding_structs_match_the_c_layout(tmp_path):
    """Every struct the binding mirrors has the size and field offsets the C
    compiler gives it from include/dmwf.h (gcc, host ABI)."""
    import shutil
    import subprocess

    from paper_1801_05358_gb300 import dmwf
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no host C compiler")
    pairs = {"dm_schedule": dmwf.DmSchedule, "dm_stats": dmwf.DmStats, "dm_profile": dmwf.DmProfile,
             "dm_server_config": dmwf.DmServerConfig, "dm_request": dmwf.DmRequest, "dm_result": dmwf.DmResult,
             "dm_server_info_t": dmwf.DmServerInfo, "dm_tuning": dmwf.DmTuning}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dmwf.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
