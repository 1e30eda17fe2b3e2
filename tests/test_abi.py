"""CPU checks of the C-ABI library: it builds, loads without a GPU, exports
every entry point include/rt3dg.h declares, and the product package never
reaches the oracle.  No compute call is made here."""
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
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            for m in re.finditer(r"^\s*(?:[\w\s\*]+?)\b(rt_\w+)\s*\(", src, flags=re.M):
                names.add(m.group(1))
    return names


def test_header_declares_entry_points():
    names = _declared()
    for must in ("rt_build_bvh", "rt_trace_visibility", "rt_trace_visibility_backward"):
        assert must in names


def test_library_builds_and_exports_everything():
    from paper_2311_16043_gb300 import _build, rt
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing
    # the binding declares exactly what the header declares
    assert set(rt.exported_symbols()) == _declared()


def test_host_only_calls():
    from paper_2311_16043_gb300 import rt
    L = rt.lib()
    assert L.rt_status_string(0) == b"ok"
    assert L.rt_status_string(1) == b"invalid argument"
    p = rt.rt_params()
    L.rt_params_default(ctypes.byref(p))
    assert p.k_sigma == 3.0 and abs(p.alpha_min - 1 / 255) < 1e-9 and abs(p.t_min - 1e-4) < 1e-9
    # invalid arguments are rejected on the host, before any device work
    out = ctypes.c_void_p()
    assert L.rt_build_bvh(None, None, None, None, -1, None, None, ctypes.byref(out)) == 1
    assert L.rt_build_bvh(None, None, None, None, 5, None, None, ctypes.byref(out)) == 1
    bad = rt.rt_params()
    L.rt_params_default(ctypes.byref(bad))
    bad.alpha_min = 1.5
    assert L.rt_build_bvh(None, None, None, None, 0, ctypes.byref(bad), None, ctypes.byref(out)) == 1
    assert L.rt_trace_visibility(None, None, None, None, None) == 1


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2311_16043_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, flags=re.M), fn
                assert "rt_oracle" not in txt, fn
