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


def test_struct_layouts_match_the_header(tmp_path):
    """Every ctypes mirror of a header struct has the C compiler's size and
    field offsets (a field added on one side only would shift the rest)."""
    import shutil
    import subprocess

    import pytest
    from paper_2010_08526_gb300 import _capi as C

    gcc = shutil.which("gcc")
    nvcc = shutil.which("nvcc")
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include") if nvcc else "/usr/local/cuda/include"
    if not gcc or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime_api.h")):
        pytest.skip("needs gcc and the CUDA headers")
    structs = {"spgemm_csc": C.SpgemmCsc, "spgemm_tuning": C.SpgemmTuning, "spgemm_opts": C.SpgemmOpts,
               "spgemm_plan_info": C.SpgemmPlanInfo, "spgemm_stats": C.SpgemmStats,
               "spgemm_allocator": C.SpgemmAllocator}
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "spgemm.h"', "int main(void) {"]
    for cname, py in structs.items():
        src.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            src.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    src.append("return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c99", "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, str(c), "-o", str(exe)],
                   check=True, capture_output=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, f"{cname}.{f}"


def test_multi_create_refuses_plan_only_options_without_gpu():
    """The multi-problem pass runs the plain plus-times product: a k-split, another
    semiring, sorted output or a prune is refused before any device call
    rather than ignored."""
    from paper_2010_08526_gb300 import _capi as C
    lib = C.load()
    dummy = ctypes.c_void_p(64)      # never dereferenced: the checks come first
    A = C.SpgemmCsc(4, 4, 0, dummy, None, None, 0, 0, 1)
    B = C.SpgemmCsc(4, 4, 0, dummy, None, None, 0, 0, 1)
    for field, value in (("kstages", 2), ("semiring", 1), ("semiring", 2), ("sort_output", 1), ("prune", 1)):
        o = C.SpgemmOpts()
        setattr(o, field, value)
        h = ctypes.c_void_p()
        st = lib.spgemm_multi_create(1, ctypes.byref(A), ctypes.byref(B), ctypes.byref(o), None, ctypes.byref(h))
        assert st == 1, (field, value)
        assert not h.value
        msg = lib.spgemm_last_error()
        assert b"k-split" in msg or b"plus-times" in msg, msg


def test_plan_create_rejects_bad_options_without_gpu():
    """Option checks run before any device call: an unknown merge mode or
    semiring, and min-plus on int64 values, are refused."""
    from paper_2010_08526_gb300 import _capi as C
    lib = C.load()
    dummy = ctypes.c_void_p(64)      # never dereferenced: the checks come first
    f32 = C.SpgemmCsc(4, 4, 0, dummy, None, None, 0, 0, 1)
    i64 = C.SpgemmCsc(4, 4, 0, dummy, None, None, 0, 0, 2)
    cases = [(f32, "merge_mode", 7, b"merge_mode"), (f32, "semiring", 9, b"semiring"),
             (i64, "semiring", 1, b"floating-point")]
    for M, field, value, word in cases:
        o = C.SpgemmOpts()
        setattr(o, field, value)
        h = ctypes.c_void_p()
        st = lib.spgemm_plan_create(ctypes.byref(M), ctypes.byref(M), ctypes.byref(o), 0, None, ctypes.byref(h))
        assert st == 1, (field, value)
        assert not h.value
        assert word in lib.spgemm_last_error(), lib.spgemm_last_error()


def test_python_option_names():
    import pytest
    from paper_2010_08526_gb300 import core
    o, _ = core._opts(semiring="or_and", merge="incremental", kstages=3)
    assert (o.semiring, o.merge_mode, o.kstages) == (2, 1, 3)
    with pytest.raises(ValueError):
        core._opts(merge="later")
    with pytest.raises(ValueError):
        core._opts(semiring="max_times")
    assert core.Tuning(hybrid_sort=True).struct().hybrid_sort == 1
    assert core.Tuning().struct().hybrid_sort == 0


def test_allocator_needs_both_callbacks_without_gpu():
    """An allocator whose free callback is NULL is refused before any device
    call (the library must be able to give back every block it takes)."""
    from paper_2010_08526_gb300 import _capi as C
    lib = C.load()
    dummy = ctypes.c_void_p(64)      # never dereferenced: the checks come first
    M = C.SpgemmCsc(4, 4, 0, dummy, None, None, 0, 0, 1)
    al = C.SpgemmAllocator(C.ALLOC_FN(lambda ctx, n, k: None), C.FREE_FN(), None)
    o = C.SpgemmOpts()
    o.allocator = ctypes.pointer(al)
    h = ctypes.c_void_p()
    st = lib.spgemm_plan_create(ctypes.byref(M), ctypes.byref(M), ctypes.byref(o), 0, None, ctypes.byref(h))
    assert st == 1 and not h.value
    assert b"allocator" in lib.spgemm_last_error()
    st = lib.spgemm_multi_create(1, ctypes.byref(M), ctypes.byref(M), ctypes.byref(o), None, ctypes.byref(h))
    assert st == 1 and not h.value
