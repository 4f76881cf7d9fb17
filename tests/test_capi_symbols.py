"""The C-ABI library loads and exports every entry point declared in include/calib.h
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "calib.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:[A-Za-z_][A-Za-z0-9_]*[\s*]+)+(calib_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_documented_entry_points():
    names = declared_functions()
    for required in ("calib_init", "calib_set_data", "calib_admm_iter", "calib_get_solutions", "calib_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1502_00858_gb300 import build, capi
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(capi.EXPORTED) == declared_functions()


def test_binding_fails_loudly_without_the_library(tmp_path):
    from paper_1502_00858_gb300 import capi
    saved = capi._lib
    capi._lib = None
    try:
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            capi.load(str(tmp_path / "missing.so"))
    finally:
        capi._lib = saved
