"""The C-ABI library loads (no GPU needed) and exports every entry point
include/boxmg.h declares, with the binding declaring the same set."""
import ctypes
import os
import re

import pytest

import paper_1803_02481_gb300 as bm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions(header="boxmg.h", prefix="bmg_"):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    pat = r"^\s*(?:int|void|long long|const char\s*\*)\s*\*?\s*(" + prefix + r"\w+)\s*\("
    return set(re.findall(pat, text, flags=re.M))


def test_header_and_binding_agree():
    names = header_functions()
    assert len(names) >= 15
    assert names == set(bm.EXPORTED), names ^ set(bm.EXPORTED)
    names3 = header_functions("boxmg3d.h", "bmg3_")
    assert len(names3) >= 7
    assert names3 == set(bm.EXPORTED3), names3 ^ set(bm.EXPORTED3)


def test_library_exports_every_declared_symbol():
    if not os.path.exists(bm.library_path()):
        from paper_1803_02481_gb300 import build
        build.build()
    cdll = ctypes.CDLL(bm.library_path())
    for name in header_functions() | header_functions("boxmg3d.h", "bmg3_"):
        assert hasattr(cdll, name), name


def test_host_only_calls_work_without_gpu():
    lib = bm.lib()
    o = bm.default_options()
    assert (o.nu1, o.nu2, o.precision, o.coarse_threshold, o.max_cycles) == (2, 1, 0, -1, 200)
    assert o.coarse_ctas == -1 and o.smoother == bm.BMG_SMOOTH_POINT
    assert lib.bmg_strerror(bm.BMG_ENOCONV).decode().startswith("no convergence")
    # argument validation happens before any device work
    h = ctypes.c_void_p()
    rc = lib.bmg_setup(None, 8, 7, ctypes.byref(o), None, ctypes.byref(h))
    assert rc == bm.BMG_EINVAL and not h.value
    rc = lib.bmg3_setup(None, 8, 7, 6, ctypes.byref(o), None, ctypes.byref(h))
    assert rc == bm.BMG_EINVAL and not h.value
    assert lib.bmg3_num_levels(None, ctypes.byref(ctypes.c_int())) == bm.BMG_EINVAL
    n = ctypes.c_int()
    assert lib.bmg_num_levels(None, ctypes.byref(n)) == bm.BMG_EINVAL
