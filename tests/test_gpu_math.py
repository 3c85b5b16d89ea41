"""The two FP64 powers the per-cell auxiliaries form by Newton's method (rho^-gamma of the
pressure sensor, the cube root of Martinelli's radius ratio) against the CUDA math library's
pow() and cbrt() on the same device, and against NumPy on the host."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ULP = np.finfo(np.float64).eps


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    # densities and radii over six decades, plus exact powers and the ends of the range
    a = 10.0 ** rng.uniform(-3, 3, n)
    b = 10.0 ** rng.uniform(-3, 3, n)
    a[:6] = [1.0, 8.0, 0.125, 1e-3, 1e3, 2.0 ** -10]
    b[:6] = [1.0, 1.0, 1.0, 1e3, 1e-3, 1.0]
    return a, b


def test_newton_powers_match_the_cuda_math_library():
    """The Newton root is the exact 7/5 power; pow(a, -1.4) raises a to the double nearest -1.4,
    8.9e-17 away from -7/5, which moves its value by |ln a| 8.9e-17 relative (up to 2.8 ulp over
    these six decades): the bound against pow() carries that term."""
    import paper_1710_04875_gb300 as P
    a, b = _inputs(1 << 16, 0)
    zn, zc, cn, cc = P.check_math(a, b)
    dp = 8.881784197001252e-17  # 7/5 - double(1.4): the double nearest 1.4 lies 8.9e-17 below it
    tol_pow = (4 * ULP + np.abs(np.log(a)) * dp) * np.abs(zc)
    assert np.all(np.abs(zn - zc) <= tol_pow), np.max(np.abs(zn - zc) / tol_pow)
    assert np.all(np.abs(cn - cc) <= 3 * ULP * np.abs(cc)), np.max(np.abs(cn / cc - 1)) / ULP
    # against the exact powers in extended precision on the host, where it has more digits
    LD = np.longdouble
    if np.finfo(LD).eps < 1e-18:
        zt = np.asarray(a, dtype=LD) ** -(LD(7) / LD(5))
        assert np.all(np.abs(np.asarray(zn, dtype=LD) - zt) <= LD(2 * ULP) * zt)
        ct = np.cbrt(np.asarray(a, dtype=LD) / np.asarray(b, dtype=LD))
        assert np.all(np.abs(np.asarray(cn, dtype=LD) - ct) <= LD(2 * ULP) * ct)
    # exact powers come out within one rounding
    for got, want in [(zn[0], 1.0), (cn[0], 1.0), (cn[1], 2.0), (cn[2], 0.5)]:
        assert abs(got - want) <= ULP * want, (got, want)
