"""The C-ABI library loads on a machine without a GPU and exports every
function that include/spgemm.h declares (no compute calls)."""
from __future__ import annotations

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "spgemm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(spgemm_[a-z_0-9]+)\s*\(", text)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_library_exports_every_declared_symbol():
    from paper_2010_08526_gb300 import build as b
    path = b.build()
    lib = ctypes.CDLL(path)
    names = header_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding declares exactly the header's functions
    from paper_2010_08526_gb300 import _capi
    assert sorted(_capi.SIGNATURES) == names


def test_version_and_error_strings_without_gpu():
    from paper_2010_08526_gb300 import _capi
    lib = _capi.load()
    assert b"sm_103a" in lib.spgemm_version()
    assert isinstance(lib.spgemm_last_error(), bytes)
    # argument checks run before any device call
    st = lib.spgemm_plan_create(None, None, None, 0, None, None)
    assert st == 1
    assert lib.spgemm_plan_destroy(None) == 0


def test_product_path_fails_loudly_without_library(tmp_path):
    from paper_2010_08526_gb300 import _capi
    import pytest
    with pytest.raises(RuntimeError):
        _capi._LIB_saved = _capi._LIB
        try:
            _capi._LIB = None
            _capi.load(str(tmp_path / "missing.so"))
        finally:
            _capi._LIB = _capi._LIB_saved
