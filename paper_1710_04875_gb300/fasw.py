"""ctypes binding of the C ABI declared in ``include/fasw.h`` (argument marshalling only).

Arrays are numpy (host) or torch CUDA tensors (device, passed by data pointer).  Every
step of the solver runs in the CUDA library; loading fails loudly if it is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

FASW_OK = 0
ERRORS = {-1: "FASW_ERR_ARG", -2: "FASW_ERR_OOM", -3: "FASW_ERR_CUDA", -4: "FASW_ERR_DIVERGED",
          -5: "FASW_ERR_DEVICE_TIMEOUT", -6: "FASW_ERR_NOT_CONVERGED", -7: "FASW_ERR_TOO_LARGE"}
FASW_AW3, FASW_AW5J, FASW_AW51, FASW_AW52, FASW_ARK3J, FASW_ARK5J, FASW_ARK51, FASW_ARK52 = range(8)
FASW_FP64, FASW_MIXED = 0, 1
KERNEL_CLASSES = ["bc", "cell_aux", "residual", "face_blocks", "diag_blocks", "sgs", "copy", "restrict",
                  "prolong", "norm", "bl"]
SCHEME_IDS = {"AW3": 0, "AW5J": 1, "AW51": 2, "AW52": 3, "ARK3J": 4, "ARK5J": 5, "ARK51": 6, "ARK52": 7}


class FaswError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = ERRORS.get(code, str(code))
        extra = ""
        if code == -3 and _lib is not None:
            extra = ": " + _lib.fasw_last_cuda_error().decode()
        super().__init__(f"{where} failed with {msg}{extra}")


class Params(C.Structure):
    _fields_ = [
        ("scheme", C.c_int), ("nlevels", C.c_int), ("gamma_cycle", C.c_int), ("nu1", C.c_int),
        ("viscous", C.c_int), ("turb", C.c_int), ("sensor", C.c_int),
        ("mach", C.c_double), ("alpha_deg", C.c_double), ("re", C.c_double), ("pr", C.c_double),
        ("prt", C.c_double), ("eta", C.c_double), ("d_cut", C.c_double), ("cfl", C.c_double),
        ("cfl_ramp", C.c_double), ("ramp_cycles", C.c_int), ("s_coarse", C.c_double),
        ("precision", C.c_int), ("norm_all", C.c_int), ("spin_limit", C.c_longlong), ("flux", C.c_int),
    ]


_lib = None
_libs: dict = {}


def library_path(variant: str = "perf") -> str:
    return _build.lib_path(variant)


def library(variant: str = "perf"):
    """Load the CUDA library (building it first when sources are newer).  variant "perf" is
    libfasw.so (FMA contraction on); "parity" is libfasw_parity.so, the same sources built
    with -fmad=false, for comparisons with a CPU reference compiled without contraction."""
    global _lib
    if variant not in _libs:
        path = _build.build(variant=variant)
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
        lib = C.CDLL(path)
        i, d, p, ll = C.c_int, C.c_double, C.c_void_p, C.c_longlong
        dp = C.c_void_p
        sig = {
            "fasw_default_params": (None, [C.POINTER(Params)]),
            "fasw_create": (i, [i, i, i, dp, dp, i, C.POINTER(Params), p, C.POINTER(p)]),
            "fasw_destroy": (None, [p]),
            "fasw_level_dims": (i, [p, i, C.POINTER(i), C.POINTER(i), C.POINTER(i)]),
            "fasw_set_state": (i, [p, i, dp, i]),
            "fasw_get_state": (i, [p, i, dp, i]),
            "fasw_set_forcing": (i, [p, i, dp, i]),
            "fasw_get_forcing": (i, [p, i, dp, i]),
            "fasw_residual": (i, [p, i, dp, dp, dp, i, C.POINTER(d)]),
            "fasw_pseudo_dt": (i, [p, i, d, dp, i]),
            "fasw_precond_apply": (i, [p, i, d, dp, dp, i]),
            "fasw_face_blocks": (i, [p, i, dp, dp, dp, dp, i]),
            "fasw_smooth": (i, [p, i, i, d]),
            "fasw_fas_cycle": (i, [p, i, C.POINTER(d)]),
            "fasw_solve_steady": (i, [p, d, i, dp, C.POINTER(i)]),
            "fasw_get_mut": (i, [p, dp, i]),
            "fasw_freeze_mut": (i, [p, dp, i]),
            "fasw_set_time_source": (i, [p, d, dp, i]),
            "fasw_launch_count": (ll, [p]),
            "fasw_profile": (i, [p, i]),
            "fasw_use_graphs": (i, [p, i]),
            "fasw_set_residual_tile": (i, [p, i]),
            "fasw_set_exact_preconditioner": (i, [p, i]),
            "fasw_set_sweep": (i, [p, i]),
            "fasw_set_motion": (i, [p, d, d, d, d]),
            "fasw_dual_time_step": (i, [p, d, i, d, i, dp, C.POINTER(i)]),
            "fasw_kernel_time": (i, [p, i, C.POINTER(ll), C.POINTER(d)]),
            "fasw_force_coefficients": (i, [p, C.POINTER(d), C.POINTER(d)]),
            "fasw_adjoint_jacobian": (i, [p, d]),
            "fasw_adjoint_set_jacobian": (i, [p, i]),
            "fasw_tangent_residual": (i, [p, dp, dp, dp, i]),
            "fasw_adjoint_apply": (i, [p, dp, dp, i, i]),
            "fasw_adjoint_objective_gradient": (i, [p, i, dp, i]),
            "fasw_adjoint_solve": (i, [p, i, dp, dp, d, i, i, d, C.POINTER(i), C.POINTER(d), i]),
            "fasw_adjoint_precond_apply": (i, [p, d, i, dp, dp, i]),
            "fasw_adjoint_set_precond_steps": (i, [p, i]),
            "fasw_adjoint_set_precond": (i, [p, i]),
            "fasw_adjoint_vertex_gradient": (i, [p, i, dp, d, dp, dp, i]),
            "fasw_adjoint_cycle_apply": (i, [p, d, i, i, dp, dp, i]),
            "fasw_adjoint_shape_gradient": (i, [p, i, dp, i, dp, d, dp, i]),
            "fasw_pitching_objective": (i, [p, d, d, d, d, d, i, i, d, i, i, C.POINTER(d), C.POINTER(i)]),
            "fasw_checkpoint_schedule": (i, [i, i, dp, dp, i, C.POINTER(i), C.POINTER(ll)]),
            "fasw_check_math": (i, [i, p, p, p, i]),
            "fasw_unsteady_adjoint": (i, [p, d, d, d, d, d, i, i, d, i, i, i, i, dp, d, d, d, i, i, d, C.POINTER(d),
                                          dp, dp, i, dp]),
            "fasw_residual_noalloc": (i, [i, i, i, dp, dp, dp, dp, C.POINTER(Params), p]),
            "fasw_batch_create": (i, [i, C.POINTER(i), C.POINTER(i), C.POINTER(i), C.POINTER(C.c_void_p),
                                      C.POINTER(C.c_void_p), i, C.POINTER(Params), p, C.POINTER(p)]),
            "fasw_batch_destroy": (None, [p]),
            "fasw_batch_case": (p, [p, i]),
            "fasw_batch_cycle": (i, [p, i, dp]),
            "fasw_batch_solve": (i, [p, d, i, dp, dp, C.POINTER(i)]),
            "fasw_batch_autotune": (i, [p, dp]),
            "fasw_batch_launch_count": (ll, [p]),
            "fasw_scheme_coefficients": (i, [i, C.POINTER(i), dp, dp]),
            "fasw_fault_inject_alloc": (None, [ll]),
            "fasw_live_allocations": (ll, []),
            "fasw_strerror": (C.c_char_p, [i]),
            "fasw_last_cuda_error": (C.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _libs[variant] = lib
        if variant == "perf":
            _lib = lib
    return _libs[variant]


def default_params(**kw) -> Params:
    p = Params()
    library().fasw_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "scheme" and isinstance(v, str):
            v = SCHEME_IDS[v]
        if k == "precision" and isinstance(v, str):
            v = {"fp64": FASW_FP64, "mixed": FASW_MIXED}[v]
        if k == "flux" and isinstance(v, str):
            v = {"jst": 0, "fvs": 1}[v]
        setattr(p, k, v)
    return p


def _check(code: int, where: str):
    if code != FASW_OK:
        raise FaswError(code, where)


def _ptr(a):
    """(pointer, on_device) of a numpy array or a torch tensor."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "need contiguous float64"
        return a.ctypes.data, 0
    # torch tensor
    assert a.is_contiguous() and str(a.dtype) == "torch.float64", "need contiguous float64 tensor"
    return a.data_ptr(), 1 if a.is_cuda else 0


class Solver:
    """One solver context on one grid; methods mirror the C entry points."""

    def __init__(self, grid, params: Params, stream=None, coords_on_device=False, variant="perf"):
        self.lib = library(variant)
        self.grid = grid
        self.params = params
        x, y = grid.coords() if not coords_on_device else grid
        self._x, self._y = x, y
        xp, xd = _ptr(x)
        yp, _ = _ptr(y)
        h = C.c_void_p()
        st = C.c_void_p(stream) if stream is not None else None
        ni, nj, nw = (grid.ni, grid.nj, grid.n_wake)
        _check(self.lib.fasw_create(ni, nj, nw, xp, yp, xd, C.byref(params), st, C.byref(h)), "fasw_create")
        self.h = h
        self.nlevels = params.nlevels
        self.finest = self.nlevels - 1

    def close(self):
        if getattr(self, "h", None):
            self.lib.fasw_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def dims(self, l):
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        _check(self.lib.fasw_level_dims(self.h, l, C.byref(a), C.byref(b), C.byref(c)), "fasw_level_dims")
        return a.value, b.value, c.value

    def _shape(self, l):
        ni, nj, _ = self.dims(l)
        return (4, nj, ni)

    def set_state(self, u, l=None):
        l = self.finest if l is None else l
        p, dev = _ptr(u)
        _check(self.lib.fasw_set_state(self.h, l, p, dev), "fasw_set_state")

    def get_state(self, l=None, out=None):
        l = self.finest if l is None else l
        out = np.zeros(self._shape(l)) if out is None else out
        p, dev = _ptr(out)
        _check(self.lib.fasw_get_state(self.h, l, p, dev), "fasw_get_state")
        return out

    def set_forcing(self, s, l):
        p, dev = _ptr(s)
        _check(self.lib.fasw_set_forcing(self.h, l, p, dev), "fasw_set_forcing")

    def get_forcing(self, l):
        out = np.zeros(self._shape(l))
        _check(self.lib.fasw_get_forcing(self.h, l, out.ctypes.data, 0), "fasw_get_forcing")
        return out

    def residual(self, l=None, want_norm=False):
        l = self.finest if l is None else l
        F = np.zeros(self._shape(l)); Fc = np.zeros_like(F); Fv = np.zeros_like(F)
        nrm = C.c_double()
        _check(self.lib.fasw_residual(self.h, l, F.ctypes.data, Fc.ctypes.data, Fv.ctypes.data, 0,
                                      C.byref(nrm) if want_norm else None), "fasw_residual")
        return (F, Fc, Fv, nrm.value) if want_norm else (F, Fc, Fv)

    def pseudo_dt(self, cfl, l=None):
        l = self.finest if l is None else l
        ni, nj, _ = self.dims(l)
        out = np.zeros((nj, ni))
        _check(self.lib.fasw_pseudo_dt(self.h, l, cfl, out.ctypes.data, 0), "fasw_pseudo_dt")
        return out

    def precond_apply(self, r, cfl, l=None):
        l = self.finest if l is None else l
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.zeros(self._shape(l))
        _check(self.lib.fasw_precond_apply(self.h, l, cfl, r.ctypes.data, z.ctypes.data, 0), "fasw_precond_apply")
        return z

    def face_blocks(self, l=None):
        l = self.finest if l is None else l
        ni, nj, _ = self.dims(l)
        axp = np.zeros((nj, ni + 1, 4, 4)); axm = np.zeros_like(axp)
        aep = np.zeros((nj + 1, ni, 4, 4)); aem = np.zeros_like(aep)
        _check(self.lib.fasw_face_blocks(self.h, l, axp.ctypes.data, axm.ctypes.data, aep.ctypes.data,
                                         aem.ctypes.data, 0), "fasw_face_blocks")
        return axp, axm, aep, aem

    def smooth(self, nsteps=1, cfl=None, l=None):
        l = self.finest if l is None else l
        cfl = self.params.cfl if cfl is None else cfl
        _check(self.lib.fasw_smooth(self.h, l, nsteps, cfl), "fasw_smooth")

    def fas_cycle(self, k: int) -> float:
        n = C.c_double()
        _check(self.lib.fasw_fas_cycle(self.h, k, C.byref(n)), "fasw_fas_cycle")
        return n.value

    def solve(self, drop: float, max_cycles: int):
        hist = np.zeros(max_cycles)
        nc = C.c_int(0)
        code = self.lib.fasw_solve_steady(self.h, drop, max_cycles, hist.ctypes.data, C.byref(nc))
        if code not in (0, -4, -6):
            _check(code, "fasw_solve_steady")
        return code, nc.value, hist[:nc.value]

    def get_mut(self):
        ni, nj, _ = self.dims(self.finest)
        out = np.zeros((nj, ni))
        _check(self.lib.fasw_get_mut(self.h, out.ctypes.data, 0), "fasw_get_mut")
        return out

    def freeze_mut(self, mut):
        """Hold the finest level's eddy viscosity at mut (nj x ni) in later cycles and solves, or
        return to the Baldwin-Lomax model (mut None)."""
        if mut is None:
            _check(self.lib.fasw_freeze_mut(self.h, None, 0), "fasw_freeze_mut")
            return
        m = np.ascontiguousarray(mut, dtype=np.float64)
        _check(self.lib.fasw_freeze_mut(self.h, m.ctypes.data, 0), "fasw_freeze_mut")

    def set_time_source(self, a_t, src=None):
        p, dev = _ptr(src)
        _check(self.lib.fasw_set_time_source(self.h, a_t, p, dev), "fasw_set_time_source")

    def launch_count(self) -> int:
        return int(self.lib.fasw_launch_count(self.h))

    def set_motion(self, phi, phidot, xc=0.25, yc=0.0):
        _check(self.lib.fasw_set_motion(self.h, phi, phidot, xc, yc), "fasw_set_motion")

    def dual_time_step(self, dt, drop, max_cycles, bdf_order=2):
        hist = np.zeros(max_cycles)
        nc = C.c_int(0)
        code = self.lib.fasw_dual_time_step(self.h, dt, bdf_order, drop, max_cycles, hist.ctypes.data, C.byref(nc))
        if code not in (0, -4, -6):
            _check(code, "fasw_dual_time_step")
        return code, nc.value, hist[:nc.value]

    def set_sweep(self, kind):
        """0 auto, 1 reference (one thread per cell), 2 one CTA, 3 strips of 8 rows, 4 strips of 16,
        5 hyperplane-staged (mixed precision), 6 / 7 staged with a ring of 4 / 8 steps, 8 strips of 4,
        9 warp strips (FP32 recurrence; FP64 contexts add one FP64 defect correction), 10 warp strips
        staging chunks of 8 steps."""
        kinds = {"auto": 0, "reference": 1, "cta": 2, "strips": 3, "strips16": 4, "staged": 5, "staged4": 6,
                 "staged8": 7, "strips4": 8, "warp": 9,
                 "warp8": 10}
        _check(self.lib.fasw_set_sweep(self.h, kinds.get(kind, kind)), "fasw_set_sweep")

    def set_exact_preconditioner(self, iters: int):
        """iters > 0: every preconditioner application iterates toward (D+L+U)^-1 (the exact
        preconditioner) by that many block Gauss-Seidel corrections; 0: the SGS preconditioner."""
        _check(self.lib.fasw_set_exact_preconditioner(self.h, int(iters)), "fasw_set_exact_preconditioner")

    def set_residual_tile(self, rows: int):
        """Residual tile height on every level: 1, 2, 4, 8, or 0 for the size rule."""
        _check(self.lib.fasw_set_residual_tile(self.h, int(rows)), "fasw_set_residual_tile")

    def use_graphs(self, enable: bool):
        _check(self.lib.fasw_use_graphs(self.h, 1 if enable else 0), "fasw_use_graphs")

    def profile(self, enable: bool):
        _check(self.lib.fasw_profile(self.h, 1 if enable else 0), "fasw_profile")

    def kernel_time(self, kernel: int):
        """(launches, total device ms) of one kernel class since profile(True)."""
        n = C.c_longlong()
        ms = C.c_double()
        _check(self.lib.fasw_kernel_time(self.h, kernel, C.byref(n), C.byref(ms)), "fasw_kernel_time")
        return n.value, ms.value

    # ---- discrete adjoint of the steady finest-level residual
    def force_coefficients(self):
        """(C_L, C_D) of the wall-face force at the current state."""
        cl, cd = C.c_double(), C.c_double()
        _check(self.lib.fasw_force_coefficients(self.h, C.byref(cl), C.byref(cd)), "fasw_force_coefficients")
        return cl.value, cd.value

    def adjoint_jacobian(self, h_rel=1e-6):
        _check(self.lib.fasw_adjoint_jacobian(self.h, h_rel), "fasw_adjoint_jacobian")

    def adjoint_set_jacobian(self, mode):
        """Jacobian assembly: "tangent" (forward-mode linearization, the default) or "differences"
        (coloured central differences)."""
        _check(self.lib.fasw_adjoint_set_jacobian(self.h, {"differences": 0, "tangent": 1}[mode]),
               "fasw_adjoint_set_jacobian")

    def tangent_residual(self, v, with_value=False):
        """(dF/du) v at the finest level's current state (and F itself with with_value)."""
        v = np.ascontiguousarray(v, dtype=np.float64)
        dF = np.zeros(self._shape(self.finest))
        F = np.zeros_like(dF) if with_value else None
        _check(self.lib.fasw_tangent_residual(self.h, v.ctypes.data, dF.ctypes.data,
                                              F.ctypes.data if with_value else None, 0), "fasw_tangent_residual")
        return (dF, F) if with_value else dF

    def adjoint_apply(self, v, transpose=False, out=None):
        v = np.ascontiguousarray(v, dtype=np.float64) if isinstance(v, np.ndarray) else v
        out = np.zeros(self._shape(self.finest)) if out is None else out
        vp, vd = _ptr(v)
        op, od = _ptr(out)
        assert vd == od, "v and out must both be host or both device"
        _check(self.lib.fasw_adjoint_apply(self.h, vp, op, 1 if transpose else 0, vd), "fasw_adjoint_apply")
        return out

    def adjoint_objective_gradient(self, which):
        out = np.zeros(self._shape(self.finest))
        _check(self.lib.fasw_adjoint_objective_gradient(self.h, which, out.ctypes.data, 0),
               "fasw_adjoint_objective_gradient")
        return out

    def adjoint_precond_apply(self, r, cfl, steps=0):
        """z = P^-T r, the transposed primal AW preconditioner scaled by eta dt* (steps 0), or that
        many steps of the primal stage loop run on J^T from zero (preconditioner kind
        "stage_loop")."""
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.zeros(self._shape(self.finest))
        _check(self.lib.fasw_adjoint_precond_apply(self.h, cfl, int(steps), r.ctypes.data, z.ctypes.data,
                                                   0),
               "fasw_adjoint_precond_apply")
        return z

    def adjoint_set_precond_steps(self, steps):
        """Smoothing steps of the transposed stage loop per GMRES preconditioner application."""
        _check(self.lib.fasw_adjoint_set_precond_steps(self.h, int(steps)), "fasw_adjoint_set_precond_steps")

    ADJOINT_PRECONDITIONERS = {"stage_loop": 0, "smoother": 1, "cycle": 2, "vcycle": 3}

    def adjoint_set_precond(self, kind):
        """Adjoint GMRES preconditioner: "stage_loop" (the stage loop run on J^T), "smoother" (the
        transposed linearised smoothing step), "cycle" (the transposed linearised FAS cycle, the
        default) or "vcycle" (the same with one coarse cycle per level).  Assemble the Jacobian
        again afterwards."""
        _check(self.lib.fasw_adjoint_set_precond(self.h, self.ADJOINT_PRECONDITIONERS[kind]),
               "fasw_adjoint_set_precond")

    def adjoint_cycle_apply(self, r, cfl, kind="cycle", transpose=True):
        """z = M r for the linear operator of the linearised smoothing step ("smoother") or FAS
        cycle ("cycle") as a solver of J, or its transpose (a solver of J^T)."""
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.zeros(self._shape(self.finest))
        _check(self.lib.fasw_adjoint_cycle_apply(self.h, cfl, self.ADJOINT_PRECONDITIONERS[kind],
                                                 1 if transpose else 0, r.ctypes.data, z.ctypes.data, 0),
               "fasw_adjoint_cycle_apply")
        return z

    def adjoint_solve(self, which=0, g=None, tol=1e-10, max_iters=400, restart=250, cfl=0.0):
        """(lam, code, iterations, relative residual) of J^T lam = g (g None: objective which);
        cfl: pseudo CFL of the preconditioner (<= 0: the parameters').  restart (<= 251) is the
        Krylov basis length, (restart + 5) x 4n doubles of device memory: short restarts stall on
        thin-layer RANS adjoints (stretched wall cells), a basis of a few hundred does not."""
        lam = np.zeros(self._shape(self.finest))
        gp = None
        if g is not None:
            g = np.ascontiguousarray(g, dtype=np.float64)
            gp = g.ctypes.data
        it, rr = C.c_int(), C.c_double()
        code = self.lib.fasw_adjoint_solve(self.h, which, gp, lam.ctypes.data, tol, max_iters, restart, cfl,
                                           C.byref(it), C.byref(rr), 0)
        if code not in (0, -6):
            _check(code, "fasw_adjoint_solve")
        return lam, code, it.value, rr.value

    def adjoint_vertex_gradient(self, which, lam, h_x=1e-6):
        """(gx, gy), each (nj+1, ni+1): dJ/dX - lam^T dF/dX for every vertex coordinate, the
        transposed product (dF/dX)^T lam with the objective's explicit part; h_x is the difference
        step relative to the shortest grid edge at each vertex."""
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        ni, nj, _ = self.dims(self.finest)
        gx = np.zeros((nj + 1, ni + 1))
        gy = np.zeros((nj + 1, ni + 1))
        _check(self.lib.fasw_adjoint_vertex_gradient(self.h, which, lam.ctypes.data, h_x, gx.ctypes.data,
                                                     gy.ctypes.data, 0), "fasw_adjoint_vertex_gradient")
        return gx, gy

    def pitching_objective(self, amp, omega, dt, nsteps, which=1, xc=0.25, yc=0.0, bdf_order=2, drop=1e-10,
                           max_cycles=500):
        """(J, code, cycles): the average of C_L (which 0) or C_D (1) over nsteps dual-time steps of the
        pitching motion alpha + amp sin(omega t), from the current state."""
        J = C.c_double()
        nc = C.c_int()
        code = self.lib.fasw_pitching_objective(self.h, amp, omega, xc, yc, dt, nsteps, bdf_order, drop, max_cycles,
                                                which, C.byref(J), C.byref(nc))
        if code not in (0, -6):
            _check(code, "fasw_pitching_objective")
        return J.value, code, nc.value

    def adjoint_shape_gradient(self, which, lam, fields, h_x=1e-6):
        """grad[k] = dJ/dX V_k - lam^T dF/dX V_k for y-displacement fields (nparam, nj+1, ni+1);
        which -1: without the objective's explicit part."""
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        V = np.ascontiguousarray(fields, dtype=np.float64)
        grad = np.zeros(V.shape[0])
        _check(self.lib.fasw_adjoint_shape_gradient(self.h, which, lam.ctypes.data, V.shape[0], V.ctypes.data, h_x,
                                                    grad.ctypes.data, 0), "fasw_adjoint_shape_gradient")
        return grad


    def unsteady_adjoint(self, amp, omega, dt, nsteps, fields=None, which=1, xc=0.25, yc=0.0, bdf_order=2,
                         drop=1e-10, max_cycles=500, snapshots=None, h_rel=1e-6, h_x=1e-6, tol=1e-10, max_iters=400,
                         restart=250, cfl=0.0):
        """Adjoint of nsteps dual-time steps of the pitching motion alpha + amp sin(omega t) from the
        current state (grid at rest): (J, dJ/dp with u^0 fixed, dJ/du^0, code, stats) with J the
        time-averaged C_L (which 0) or C_D (1), p the amplitudes of the y-displacement fields
        (nparam, nj+1, ni+1), and stats = {forward_steps, recomputed_steps, gmres_iterations,
        cycles, worst_relative_residual}.  snapshots: stored time levels for the reverse sweep
        (None: every level)."""
        V = np.zeros((0,)) if fields is None else np.ascontiguousarray(fields, dtype=np.float64)
        nparam = 0 if fields is None else V.shape[0]
        snaps = nsteps if snapshots is None else int(snapshots)
        J = C.c_double()
        grad = np.zeros(max(nparam, 1))
        g0 = np.zeros(self._shape(self.finest))
        st = np.zeros(5)
        code = self.lib.fasw_unsteady_adjoint(self.h, amp, omega, xc, yc, dt, nsteps, bdf_order, drop, max_cycles,
                                              snaps, which, nparam, V.ctypes.data if nparam else None, h_rel, h_x,
                                              tol, max_iters, restart, cfl, C.byref(J), grad.ctypes.data,
                                              g0.ctypes.data, 0, st.ctypes.data)
        if code not in (0, -6):
            _check(code, "fasw_unsteady_adjoint")
        stats = {"forward_steps": int(st[0]), "recomputed_steps": int(st[1]), "gmres_iterations": int(st[2]),
                 "cycles": int(st[3]), "worst_relative_residual": float(st[4])}
        return J.value, grad[:nparam], g0, code, stats


def checkpoint_schedule(nsteps, snapshots):
    """(actions, forward_steps) of the binomial checkpoint schedule for the reverse sweep of the
    unsteady adjoint: actions are (op, level) pairs, op 0 advance to, 1 store, 2 restore,
    3 adjoint step, 4 free (host code; no GPU needed)."""
    lib = library()
    n = C.c_int()
    fs = C.c_longlong()
    _check(lib.fasw_checkpoint_schedule(nsteps, snapshots, None, None, 0, C.byref(n), C.byref(fs)),
           "fasw_checkpoint_schedule")
    ops = np.zeros(n.value, dtype=np.int32)
    args = np.zeros(n.value, dtype=np.int32)
    _check(lib.fasw_checkpoint_schedule(nsteps, snapshots, ops.ctypes.data, args.ctypes.data, n.value, C.byref(n),
                                        C.byref(fs)), "fasw_checkpoint_schedule")
    return list(zip(ops.tolist(), args.tolist())), fs.value


def check_math(a, b):
    """(rho^-gamma by Newton, pow(a, -gamma), (a/b)^(1/3) by Newton, cbrt(a/b)) per element, each an
    array like a: the library's FP64 powers beside the CUDA math library's, on the current GPU."""
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    b = np.ascontiguousarray(b, dtype=np.float64).ravel()
    if a.shape != b.shape:
        raise ValueError("a and b differ in size")
    out = np.zeros((a.size, 4))
    _check(library().fasw_check_math(a.size, a.ctypes.data, b.ctypes.data, out.ctypes.data, 0), "fasw_check_math")
    return out[:, 0], out[:, 1], out[:, 2], out[:, 3]


class Batch:
    """Many independent cases advanced together (one captured CUDA graph per cycle)."""

    def __init__(self, grids, params_list, stream=None):
        self.lib = library()
        n = len(grids)
        self.grids = grids
        self._coords = [g.coords() for g in grids]
        ni = (C.c_int * n)(*[g.ni for g in grids])
        nj = (C.c_int * n)(*[g.nj for g in grids])
        nw = (C.c_int * n)(*[g.n_wake for g in grids])
        xs = (C.c_void_p * n)(*[c[0].ctypes.data for c in self._coords])
        ys = (C.c_void_p * n)(*[c[1].ctypes.data for c in self._coords])
        self.params = list(params_list)
        ps = (Params * n)(*params_list)
        h = C.c_void_p()
        st = C.c_void_p(stream) if stream is not None else None
        _check(self.lib.fasw_batch_create(n, ni, nj, nw, xs, ys, 0, ps, st, C.byref(h)), "fasw_batch_create")
        self.h = h
        self.n = n

    def close(self):
        if getattr(self, "h", None):
            self.lib.fasw_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def cycle(self, k):
        norms = np.zeros(self.n)
        _check(self.lib.fasw_batch_cycle(self.h, k, norms.ctypes.data), "fasw_batch_cycle")
        return norms

    def solve(self, drop, max_cycles):
        cyc = np.zeros(self.n, dtype=np.float64)
        fd = np.zeros(self.n)
        ncy = C.c_int(0)
        ci = (C.c_int * self.n)()
        code = self.lib.fasw_batch_solve(self.h, drop, max_cycles, C.cast(ci, C.c_void_p), fd.ctypes.data,
                                         C.byref(ncy))
        if code not in (0, -4, -6):
            _check(code, "fasw_batch_solve")
        return code, np.array(list(ci)), fd, ncy.value

    def autotune(self, with_tiles=False):
        """Sweep kind per case (with_tiles: (kind, residual tile height) per case)."""
        ch = (C.c_int * self.n)()
        _check(self.lib.fasw_batch_autotune(self.h, C.cast(ch, C.c_void_p)), "fasw_batch_autotune")
        if with_tiles:
            return [(x & 0xFF, x >> 8) for x in ch]
        return [x & 0xFF for x in ch]

    def get_state(self, k):
        g = self.grids[k]
        out = np.zeros((4, g.nj, g.ni))
        ctx = self.lib.fasw_batch_case(self.h, k)
        _check(self.lib.fasw_get_state(ctx, self.params[k].nlevels - 1, out.ctypes.data, 0), "fasw_get_state")
        return out

    def launch_count(self):
        return int(self.lib.fasw_batch_launch_count(self.h))
