"""Python handle on the FP64 CPU oracle (``fasw_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py``; never by the product
package.  The oracle shares no code with the CUDA library.

The coefficient table below is the paper's Table "RK smoothers" (section 4.1),
with the readings G15/G16/G18: AW3 uses the ARK3J coefficients, the 5-stage W
methods AW51/AW52 use the ARK51/ARK52 alphas with the ARK5J betas, and the
ARK5J beta row is read as (1, 0, 0.56, 0, 0.44).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fasw_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libfasw_oracle.so")

# Table "RK smoothers": alpha_i, beta_i
SCHEMES = {
    "ARK3J": ((0.1481, 2.0 / 5.0, 1.0), (1.0, 0.5, 0.5)),
    "ARK5J": ((1.0 / 4.0, 1.0 / 6.0, 3.0 / 8.0, 1.0 / 2.0, 1.0), (1.0, 0.0, 0.56, 0.0, 0.44)),
    "ARK51": ((0.0533, 0.1263, 0.2375, 0.4414, 1.0), (1.0, 0.0, 0.56, 0.0, 0.44)),
    "ARK52": ((0.0695, 0.1602, 0.2898, 0.5060, 1.0), (1.0, 0.0, 0.56, 0.0, 0.44)),
}
SCHEMES["ERK3J"] = (SCHEMES["ARK3J"][0], (1.0, 1.0, 1.0))   # beta = 1: unsplit (section 4.1)
SCHEMES["W3"] = SCHEMES["ERK3J"]
SCHEMES["AW3"] = SCHEMES["ARK3J"]
SCHEMES["AW5J"] = SCHEMES["ARK5J"]
SCHEMES["AW51"] = SCHEMES["ARK51"]
SCHEMES["AW52"] = SCHEMES["ARK52"]


class OrParams(C.Structure):
    _fields_ = [
        ("scheme", C.c_int), ("nstages", C.c_int),
        ("alpha", C.c_double * 5), ("beta", C.c_double * 5),
        ("nlevels", C.c_int), ("gamma_cycle", C.c_int), ("nu1", C.c_int),
        ("viscous", C.c_int), ("turb", C.c_int), ("sensor", C.c_int),
        ("mach", C.c_double), ("alpha_deg", C.c_double), ("re", C.c_double),
        ("pr", C.c_double), ("prt", C.c_double),
        ("eta", C.c_double), ("d_cut", C.c_double), ("cfl", C.c_double),
        ("cfl_ramp", C.c_double), ("ramp_cycles", C.c_int),
        ("s_coarse", C.c_double), ("dt_phys", C.c_double), ("bdf_order", C.c_int),
        ("norm_all", C.c_int), ("flux", C.c_int), ("precond", C.c_int),
    ]


# Two builds of the same source: "parity" (the reference the tests compare with: no FMA
# contraction, -O2) and "timing" (the CPU baseline the benchmark times: -O3 with contraction
# allowed; the same arithmetic up to rounding, no machine-specific flags so that it builds the
# same on x86 and Arm hosts).
_FLAGS = {"parity": ["-O2", "-ffp-contract=off"], "timing": ["-O3", "-ffp-contract=fast"]}
_LIBS = {"parity": _LIB, "timing": os.path.join(_HERE, "_build", "libfasw_oracle_timing.so")}


def build(force: bool = False, variant: str = "parity") -> str:
    """Compile one build of the oracle with g++ (see _FLAGS)."""
    out = _LIBS[variant]
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", *_FLAGS[variant], "-std=c++17", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, out)
    return out


def build_all(force: bool = False):
    return [build(force, v) for v in _FLAGS]


_libs: dict = {}


def lib(variant: str = "parity"):
    if variant not in _libs:
        _lib = C.CDLL(build(variant=variant))
        d, i, p = C.c_double, C.c_int, C.c_void_p
        dp = C.POINTER(C.c_double)
        sig = {
            "or_create": (p, [i, i, i, dp, dp, C.POINTER(OrParams)]),
            "or_destroy": (None, [p]),
            "or_free_stream": (None, [d, d, dp]),
            "or_nlevels": (i, [p]),
            "or_level_dims": (None, [p, i, C.POINTER(i), C.POINTER(i), C.POINTER(i)]),
            "or_get_metrics": (None, [p, i, dp, dp, dp, dp, dp]),
            "or_set_state": (None, [p, i, dp]),
            "or_get_state": (None, [p, i, dp]),
            "or_get_ghosted": (None, [p, i, dp]),
            "or_set_forcing": (None, [p, i, dp]),
            "or_get_forcing": (None, [p, i, dp]),
            "or_set_mut": (None, [p, i, dp]),
            "or_get_mut": (None, [p, i, dp]),
            "or_compute_mut": (None, [p]),
            "or_residual": (None, [p, i, dp, dp, dp]),
            "or_wall_force": (None, [p, dp, dp]),
            "or_pseudo_dt": (None, [p, i, d, dp]),
            "or_precond_apply": (None, [p, i, d, dp, dp, i, dp]),
            "or_face_blocks": (None, [p, i, dp, dp, dp, dp]),
            "or_smooth": (None, [p, i, i, d, i]),
            "or_fas_cycle": (d, [p, i]),
            "or_solve": (i, [p, d, i, dp]),
            "or_set_time_source": (None, [p, d, dp]),
            "or_conv_flux": (None, [dp, d, d, dp]),
            "or_split_jacobians": (None, [dp, d, d, d, dp, dp]),
            "or_eigvecs": (None, [dp, d, d, dp, dp]),
            "or_cutoff": (d, [d, d, d]),
            "or_sensor": (d, [d, d, d]),
            "or_farfield_state": (None, [dp, dp, d, d, dp]),
            "or_stage_scalar": (d, [i, dp, dp, d, d, d, d]),
            "or_restrict": (None, [p, i, dp, dp]),
            "or_prolong": (None, [p, i, dp, dp]),
            "or_linear_step": (None, [dp, d, d, i, i, d, d, d, d, i, i, i, dp, dp, dp, dp, dp, dp]),
            "or_set_motion": (None, [p, d, d, d, d]),
            "or_dual_time_step": (i, [p, d, d, i, dp]),
            "or_grid_fluxes": (None, [p, i, dp, dp]),
            "or_block_apply": (None, [p, i, d, dp, dp]),
            "or_residual_complex_step": (None, [p, i, dp, d, dp, dp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
        _libs[variant] = _lib
    return _libs[variant]


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_params(scheme: str = "AW3", nlevels: int = 3, gamma_cycle: int = 1, nu1: int = 1,
                viscous: int = 0, turb: int = 0, sensor: int | None = None, mach: float = 0.8,
                alpha_deg: float = 0.0, re: float = 1e6, pr: float = 0.75, prt: float = 0.9,
                eta: float = 0.8, d_cut: float = 0.5, cfl: float = 1e4, cfl_ramp: float = 20.0,
                ramp_cycles: int = 2, s_coarse: float = 0.25, dt_phys: float = 0.0,
                bdf_order: int = 2, norm_all: int = 0, flux: str = "jst", precond: str = "sgs") -> OrParams:
    al, be = SCHEMES[scheme]
    p = OrParams()
    p.scheme = 1 if (scheme.startswith("ARK") or scheme.startswith("ERK")) else 0
    p.nstages = len(al)
    for k in range(5):
        p.alpha[k] = al[k] if k < len(al) else 0.0
        p.beta[k] = be[k] if k < len(be) else 0.0
    p.nlevels, p.gamma_cycle, p.nu1 = nlevels, gamma_cycle, nu1
    p.viscous, p.turb = viscous, turb
    p.sensor = (1 if viscous else 0) if sensor is None else sensor
    p.mach, p.alpha_deg, p.re, p.pr, p.prt = mach, alpha_deg, re, pr, prt
    p.eta, p.d_cut, p.cfl, p.cfl_ramp, p.ramp_cycles = eta, d_cut, cfl, cfl_ramp, ramp_cycles
    p.s_coarse, p.dt_phys, p.bdf_order, p.norm_all = s_coarse, dt_phys, bdf_order, norm_all
    p.flux = {"jst": 0, "fvs": 1}[flux]
    p.precond = {"sgs": 0, "exact": 1}[precond]
    return p


class Oracle:
    """One oracle solver instance on a C-grid (all levels)."""

    def __init__(self, grid, params: OrParams, variant: str = "parity"):
        self.L = lib(variant)
        self.grid = grid
        self.params = params
        x, y = grid.coords()
        self._x, self._y = x, y
        self.h = self.L.or_create(grid.ni, grid.nj, grid.n_wake, _dp(x), _dp(y), C.byref(params))
        if not self.h:
            raise ValueError("oracle rejected the grid/parameters")
        self.nlevels = self.L.or_nlevels(self.h)
        self.finest = self.nlevels - 1

    def __del__(self):
        if getattr(self, "h", None):
            self.L.or_destroy(self.h)
            self.h = None

    def dims(self, l: int):
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        self.L.or_level_dims(self.h, l, C.byref(a), C.byref(b), C.byref(c))
        return a.value, b.value, c.value

    def n(self, l):
        ni, nj, _ = self.dims(l)
        return ni * nj

    def metrics(self, l):
        ni, nj, _ = self.dims(l)
        sxx = np.zeros((nj, ni + 1)); sxy = np.zeros((nj, ni + 1))
        sex = np.zeros((nj + 1, ni)); sey = np.zeros((nj + 1, ni))
        vol = np.zeros((nj, ni))
        self.L.or_get_metrics(self.h, l, _dp(sxx), _dp(sxy), _dp(sex), _dp(sey), _dp(vol))
        return sxx, sxy, sex, sey, vol

    def set_state(self, u, l=None):
        l = self.finest if l is None else l
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.size == 4 * self.n(l)
        self.L.or_set_state(self.h, l, _dp(u))

    def get_state(self, l=None):
        l = self.finest if l is None else l
        ni, nj, _ = self.dims(l)
        u = np.zeros((4, nj, ni))
        self.L.or_get_state(self.h, l, _dp(u))
        return u

    def ghosted(self, l=None):
        l = self.finest if l is None else l
        ni, nj, _ = self.dims(l)
        u = np.zeros((4, nj + 4, ni + 4))
        self.L.or_get_ghosted(self.h, l, _dp(u))
        return u

    def set_forcing(self, s, l):
        s = np.ascontiguousarray(s, dtype=np.float64)
        self.L.or_set_forcing(self.h, l, _dp(s))

    def get_forcing(self, l):
        ni, nj, _ = self.dims(l)
        s = np.zeros((4, nj, ni))
        self.L.or_get_forcing(self.h, l, _dp(s))
        return s

    def set_mut(self, m, l=None):
        l = self.finest if l is None else l
        m = np.ascontiguousarray(m, dtype=np.float64)
        self.L.or_set_mut(self.h, l, _dp(m))

    def get_mut(self, l=None):
        l = self.finest if l is None else l
        ni, nj, _ = self.dims(l)
        m = np.zeros((nj, ni))
        self.L.or_get_mut(self.h, l, _dp(m))
        return m

    def compute_mut(self):
        self.L.or_compute_mut(self.h)
        return self.get_mut()

    def residual(self, l=None):
        """(F, F^c, F^v), each (4, nj, ni), per unit volume."""
        l = self.finest if l is None else l
        ni, nj, _ = self.dims(l)
        F = np.zeros((4, nj, ni)); Fc = np.zeros_like(F); Fv = np.zeros_like(F)
        self.L.or_residual(self.h, l, _dp(F), _dp(Fc), _dp(Fv))
        return F, Fc, Fv

    def residual_complex_step(self, v, h=1e-30, l=None):
        """(F, dF): the residual and its directional derivative (dF/du) v by the complex step
        (the residual's formulas evaluated at u + i h v; Im / h has no differencing error).  The
        eddy viscosity is held at its current value.  v: (4, nj, ni)."""
        l = self.finest if l is None else l
        ni, nj, _ = self.dims(l)
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(4, nj, ni)
        F = np.zeros((4, nj, ni)); dF = np.zeros_like(F)
        self.L.or_residual_complex_step(self.h, l, _dp(v), h, _dp(F), _dp(dF))
        return F, dF

    def wall_force(self):
        """Per-wall-face force on the body (fx, fy), ni entries each (zero on the wake cut), from
        the residual's own j = 0 face fluxes at the current state (finest level)."""
        ni = self.grid.ni
        fx = np.zeros(ni); fy = np.zeros(ni)
        self.L.or_wall_force(self.h, _dp(fx), _dp(fy))
        return fx, fy

    def pseudo_dt(self, cfl, l=None):
        l = self.finest if l is None else l
        ni, nj, _ = self.dims(l)
        d = np.zeros((nj, ni))
        self.L.or_pseudo_dt(self.h, l, cfl, _dp(d))
        return d

    def block_apply(self, x, cfl, l=None):
        """(D + L + U) x with the blocks at the level's current state."""
        l = self.finest if l is None else l
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros_like(x)
        self.L.or_block_apply(self.h, l, cfl, _dp(x), _dp(y))
        return y

    def precond_apply(self, r, cfl, l=None, dense=False):
        l = self.finest if l is None else l
        ni, nj, _ = self.dims(l)
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.zeros((4, nj, ni))
        D = np.zeros((nj * ni, 4, 4))
        mode = 2 if dense == "exact" else (1 if dense else 0)   # "exact": (D + L + U)^-1
        self.L.or_precond_apply(self.h, l, cfl, _dp(r), _dp(z), mode, _dp(D))
        return z, D

    def face_blocks(self, l=None):
        l = self.finest if l is None else l
        ni, nj, _ = self.dims(l)
        axp = np.zeros((nj, ni + 1, 4, 4)); axm = np.zeros_like(axp)
        aep = np.zeros((nj + 1, ni, 4, 4)); aem = np.zeros_like(aep)
        self.L.or_face_blocks(self.h, l, _dp(axp), _dp(axm), _dp(aep), _dp(aem))
        return axp, axm, aep, aem

    def smooth(self, nsteps=1, cfl=None, l=None, dense=False):
        l = self.finest if l is None else l
        cfl = self.params.cfl if cfl is None else cfl
        self.L.or_smooth(self.h, l, nsteps, cfl, 1 if dense else 0)

    def fas_cycle(self, k: int) -> float:
        return self.L.or_fas_cycle(self.h, k)

    def solve(self, drop: float, max_cycles: int):
        hist = np.zeros(max_cycles)
        nc = self.L.or_solve(self.h, drop, max_cycles, _dp(hist))
        return nc, hist[:abs(nc)]

    def set_time_source(self, a_t: float, src=None):
        if src is None:
            self.L.or_set_time_source(self.h, a_t, None)
        else:
            src = np.ascontiguousarray(src, dtype=np.float64)
            self.L.or_set_time_source(self.h, a_t, _dp(src))

    def set_motion(self, phi, phidot, xc=0.25, yc=0.0):
        self.L.or_set_motion(self.h, phi, phidot, xc, yc)

    def dual_time_step(self, dt, drop, max_cycles):
        hist = np.zeros(max_cycles)
        nc = self.L.or_dual_time_step(self.h, dt, drop, max_cycles, _dp(hist))
        return nc, hist[:abs(nc)]

    def grid_fluxes(self, l=None):
        l = self.finest if l is None else l
        ni, nj, _ = self.dims(l)
        vfx = np.zeros((nj, ni + 1)); vfe = np.zeros((nj + 1, ni))
        self.L.or_grid_fluxes(self.h, l, _dp(vfx), _dp(vfe))
        return vfx, vfe

    def restrict(self, l, vf):
        vf = np.ascontiguousarray(vf, dtype=np.float64)
        ni, nj, _ = self.dims(l - 1)
        vc = np.zeros((4, nj, ni))
        self.L.or_restrict(self.h, l, _dp(vf), _dp(vc))
        return vc

    def prolong(self, l, dc):
        dc = np.ascontiguousarray(dc, dtype=np.float64)
        ni, nj, _ = self.dims(l)
        df = np.zeros((4, nj, ni))
        self.L.or_prolong(self.h, l, _dp(dc), _dp(df))
        return df


# ---- point functions
def free_stream(mach, alpha_deg):
    out = np.zeros(4)
    lib().or_free_stream(mach, alpha_deg, _dp(out))
    return out


def conv_flux(w, sx, sy):
    w = np.ascontiguousarray(w, dtype=np.float64); f = np.zeros(4)
    lib().or_conv_flux(_dp(w), sx, sy, _dp(f))
    return f


def split_jacobians(w, sx, sy, d):
    w = np.ascontiguousarray(w, dtype=np.float64)
    Ap = np.zeros((4, 4)); Am = np.zeros((4, 4))
    lib().or_split_jacobians(_dp(w), sx, sy, d, _dp(Ap), _dp(Am))
    return Ap, Am


def eigvecs(w, nx, ny):
    w = np.ascontiguousarray(w, dtype=np.float64)
    R = np.zeros((4, 4)); Ri = np.zeros((4, 4))
    lib().or_eigvecs(_dp(w), nx, ny, _dp(R), _dp(Ri))
    return R, Ri


def cutoff(lam, a, d):
    return lib().or_cutoff(lam, a, d)


def sensor(qm, q0, qp):
    return lib().or_sensor(qm, q0, qp)


def farfield_state(wi, winf, nx, ny):
    wi = np.ascontiguousarray(wi, dtype=np.float64)
    winf = np.ascontiguousarray(winf, dtype=np.float64)
    out = np.zeros(4)
    lib().or_farfield_state(_dp(wi), _dp(winf), nx, ny, _dp(out))
    return out


def stage_scalar(scheme, lc, lv, dts, w):
    al, be = SCHEMES[scheme]
    a = np.zeros(5); b = np.zeros(5)
    a[:len(al)] = al; b[:len(be)] = be
    return lib().or_stage_scalar(len(al), _dp(a), _dp(b), lc, lv, dts, w)


def linear_step(w, dx, dy, nx, ny, u, dts, eta=0.8, a_t=0.0, d=0.5, scheme="AW3", circulant=True):
    """One smoothing step of the linear model (section 5) on u (4, ny, nx); returns (u_new, A, B, M)."""
    al, be = SCHEMES[scheme]
    a = np.zeros(5); b = np.zeros(5)
    a[:len(al)] = al; b[:len(be)] = be
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.ascontiguousarray(u, dtype=np.float64).copy()
    A = np.zeros((4, 4)); B = np.zeros((4, 4)); M = np.zeros((4, 4))
    aw = 0 if (scheme.startswith("ARK") or scheme.startswith("ERK")) else 1
    lib().or_linear_step(_dp(w), dx, dy, nx, ny, dts, eta, a_t, d, aw, 1 if circulant else 0, len(al),
                         _dp(a), _dp(b), _dp(out), _dp(A), _dp(B), _dp(M))
    return out, A, B, M
