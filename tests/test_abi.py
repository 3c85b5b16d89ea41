"""CPU checks of the C ABI boundary: the library builds/loads and exports every
declared entry point; no compute call is made without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "fasw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fasw_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["fasw_create", "fasw_destroy", "fasw_residual", "fasw_smooth", "fasw_fas_cycle",
                     "fasw_solve_steady", "fasw_set_time_source", "fasw_set_state", "fasw_get_state"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_1710_04875_gb300 as P
    lib = ctypes.CDLL(P.library_path() if os.path.exists(P.library_path()) else P.fasw._build.build())
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_params_and_strerror_are_host_only():
    import paper_1710_04875_gb300 as P
    p = P.default_params()
    assert p.scheme == P.FASW_AW3 and p.nlevels == 3 and abs(p.eta - 0.8) < 1e-15 and p.d_cut == 0.5
    lib = P.library()
    assert lib.fasw_strerror(-4) == b"residual diverged"


def test_check_math_rejects_bad_arguments_before_touching_the_device():
    import paper_1710_04875_gb300 as P
    lib = P.library()
    assert lib.fasw_check_math(-1, None, None, None, 0) == -1
    assert lib.fasw_check_math(4, None, None, None, 0) == -1
    assert lib.fasw_check_math(0, None, None, None, 0) == 0


def test_create_rejects_bad_arguments_before_touching_the_device():
    import paper_1710_04875_gb300 as P
    from synth.cgrid import make_cgrid
    g = make_cgrid(32, 8)
    lib = P.library()
    x, y = g.coords()
    h = ctypes.c_void_p()
    p = P.default_params(nlevels=5)          # 32/16 = 2 < 4 coarsest cells in i
    rc = lib.fasw_create(32, 8, 4, x.ctypes.data, y.ctypes.data, 0, ctypes.byref(p), None, ctypes.byref(h))
    assert rc == -1
    p = P.default_params(nlevels=2)
    rc = lib.fasw_create(33, 8, 4, x.ctypes.data, y.ctypes.data, 0, ctypes.byref(p), None, ctypes.byref(h))
    assert rc == -1
    rc = lib.fasw_create(32, 8, 4, None, y.ctypes.data, 0, ctypes.byref(p), None, ctypes.byref(h))
    assert rc == -1


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1710_04875_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text and "fasw_oracle" not in text, f


def test_noalloc_rejects_oversized_dimensions_before_touching_the_device():
    """Sizes whose int products would overflow are rejected from 64-bit arithmetic on the raw
    sizes, before any pointer is used (host arrays stand in for the device pointers here)."""
    import numpy as np
    import paper_1710_04875_gb300 as P
    lib = P.library()
    p = P.default_params(nlevels=1)
    buf = np.zeros(16)
    ptr = buf.ctypes.data
    for ni, nj in [(1 << 20, 1 << 20), (2**31 - 1, 4), (4, 2**31 - 1), (70000, 70000), (512, 128)]:
        nw = ni // 8
        rc = lib.fasw_residual_noalloc(ni, nj, nw, ptr, ptr, ptr, ptr, ctypes.byref(p), None)
        assert rc == -7, (ni, nj, rc)
    assert lib.fasw_residual_noalloc(64, 16, 2**31 - 1, ptr, ptr, ptr, ptr, ctypes.byref(p), None) == -1


def test_scheme_coefficients_and_fault_injection_are_host_only():
    import paper_1710_04875_gb300 as P
    lib = P.library()
    lib.fasw_live_allocations.restype = ctypes.c_longlong
    lib.fasw_fault_inject_alloc.argtypes = [ctypes.c_longlong]
    assert lib.fasw_live_allocations() >= 0
    lib.fasw_fault_inject_alloc(-1)
    ns = ctypes.c_int()
    assert lib.fasw_scheme_coefficients(0, ctypes.byref(ns), None, None) == 0 and ns.value == 3
