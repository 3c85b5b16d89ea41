"""The stage coefficients of Table "RK smoothers" (section 4.1), read from the golden file
that transcribes the paper, against both tables that use them: the oracle's SCHEMES and the
CUDA library's own table (queried through the C ABI, host only).  The two are written out
independently, so a typo in either fails here; the schemes the paper derives (W methods with
the ARK coefficients of the same name, the 5-stage 1/2 schemes with the ARK5J betas, the
ARK5J beta row read as 1, 0, 0.56, 0, 0.44) are checked as the paper states them."""
import ctypes
import json
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def table():
    return json.load(open(GOLDEN))["rk_coefficients"]


def expected(name):
    """(alpha, beta) of a scheme as the paper defines it: AWx takes ARKx's coefficients, and
    ARK51/ARK52 (not additive in their origin) take ARK5J's betas."""
    t = table()
    # AW3 is the W method of ARK3J (reading G18: the paper never prints AW3's coefficients)
    base = {"AW3": "ARK3J"}.get(name, "ARK" + name[2:] if name.startswith("AW") else name)
    alpha = t[base]["alpha"]
    beta = t[base].get("beta", t["ARK5J"]["beta"])
    return alpha, beta


SCHEMES = ["AW3", "AW5J", "AW51", "AW52", "ARK3J", "ARK5J", "ARK51", "ARK52"]


def test_golden_table_is_the_printed_one():
    t = table()
    assert t["ARK3J"]["alpha"] == [0.1481, 0.4, 1.0] and t["ARK3J"]["beta"] == [1.0, 0.5, 0.5]
    assert np.allclose(t["ARK5J"]["alpha"], [1 / 4, 1 / 6, 3 / 8, 1 / 2, 1], rtol=0, atol=1e-16)
    assert t["ARK5J"]["beta"] == [1.0, 0.0, 0.56, 0.0, 0.44]
    # a consistent additive scheme: the betas of each scheme sum to one in the blending
    # recursion f_i = beta_i g_i + (1 - beta_i) f_(i-1) with beta_1 = 1
    for k in ("ARK3J", "ARK5J"):
        assert t[k]["beta"][0] == 1.0
    # every scheme's last stage is the full step
    for k in ("ARK3J", "ARK5J", "ARK51", "ARK52"):
        assert t[k]["alpha"][-1] == 1.0


@pytest.mark.parametrize("name", SCHEMES)
def test_oracle_coefficients_are_the_papers(name):
    alpha, beta = expected(name)
    a, b = O.SCHEMES[name]
    assert list(a) == pytest.approx(alpha, abs=1e-16)
    assert list(b) == pytest.approx(beta, abs=1e-16)


@pytest.mark.parametrize("name", SCHEMES)
def test_library_coefficients_are_the_papers(name):
    import paper_1710_04875_gb300 as P
    lib = P.library()
    lib.fasw_scheme_coefficients.restype = ctypes.c_int
    lib.fasw_scheme_coefficients.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p,
                                             ctypes.c_void_p]
    ns = ctypes.c_int()
    a = np.zeros(5)
    b = np.zeros(5)
    assert lib.fasw_scheme_coefficients(P.SCHEME_IDS[name], ctypes.byref(ns), a.ctypes.data, b.ctypes.data) == 0
    alpha, beta = expected(name)
    assert ns.value == len(alpha)
    assert list(a[:ns.value]) == pytest.approx(alpha, abs=1e-16)
    assert list(b[:ns.value]) == pytest.approx(beta, abs=1e-16)
    assert lib.fasw_scheme_coefficients(8, ctypes.byref(ns), None, None) == -1


def test_a_planted_typo_in_the_table_is_caught():
    """The check above is not vacuous: one digit changed in a copy of a scheme fails it."""
    alpha, beta = expected("ARK51")
    typo = list(alpha)
    typo[2] = 0.2357
    assert list(typo) != pytest.approx(alpha, abs=1e-16)
