"""FP64 CPU oracle of the explicit phase-field PVD step (arXiv 2312.05410).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path never
imports this package.  It shares no code with the CUDA path; both start from
the arrays made by ``paper_2312_05410_gb300.inputs``.

The arithmetic lives in ``pf_oracle.c`` (plain loops, one ghost ring, double
precision); this module compiles it with gcc on first use and marshals numpy
arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pf_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")  # the same loops over all host cores
_lock = threading.Lock()
_lib = None


class OrcParams(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "dx", "dt", "W_c", "W_phi", "kappa_c", "kappa_phi",
        "MA_bulk", "MB_bulk", "MA_surf", "MB_surf", "sigma_surf",
        "M_phi", "L_phi", "D_rho", "v_mag", "v_angle_deg", "rho_top")] + [
        ("phi_mode", C.c_int), ("deposition", C.c_int), ("diag_every", C.c_int)]


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle: plain -O2, single thread (the checker); with openmp=True the same source
    with -fopenmp into a second library (the all-cores CPU baseline)."""
    out = _LIB_OMP if openmp else _LIB
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        flags = ["-fopenmp"] if openmp else []
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", *flags, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def _bind(L):
    dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
    P = C.POINTER(OrcParams)
    L.orc_step.argtypes = [P, C.c_int, C.c_int, dp, dp, dp, C.c_long]
    L.orc_step.restype = C.c_int
    return L


_lib_omp = None


def lib_omp():
    """The -fopenmp build (CPU baseline only: the checker is lib())."""
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            _lib_omp = _bind(C.CDLL(build(openmp=True)))
    return _lib_omp


def step_all_cores(pd, phi, c, rho, nsteps: int):
    """O.step through the OpenMP build (identical results, rows split over the host's cores)."""
    phi, c, rho = _f64(phi).copy(), _f64(c).copy(), _f64(rho).copy()
    ny, nx = phi.shape
    rc = lib_omp().orc_step(C.byref(params(pd)), nx, ny, phi, c, rho, int(nsteps))
    assert rc == 0
    return phi, c, rho


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
            P = C.POINTER(OrcParams)
            for name in ("orc_p", "orc_dp", "orc_h", "orc_g", "orc_dg"):
                f = getattr(L, name)
                f.argtypes, f.restype = [C.c_double], C.c_double
            L.orc_f.argtypes, L.orc_f.restype = [P, C.c_double, C.c_double], C.c_double
            L.orc_mobility.argtypes, L.orc_mobility.restype = [P, C.c_double, C.c_double], C.c_double
            L.orc_chem_pot.argtypes = [P, C.c_int, C.c_int, dp, dp, dp, dp]
            L.orc_chem_pot.restype = C.c_int
            L.orc_rhs.argtypes = [P, C.c_int, C.c_int, dp, dp, dp, dp, dp, dp]
            L.orc_rhs.restype = C.c_int
            L.orc_step.argtypes = [P, C.c_int, C.c_int, dp, dp, dp, C.c_long]
            L.orc_step.restype = C.c_int
            L.orc_free_energy.argtypes, L.orc_free_energy.restype = [P, C.c_int, C.c_int, dp, dp], C.c_double
            L.orc_diag.argtypes, L.orc_diag.restype = [P, C.c_int, C.c_int, dp, dp, dp, dp], None
            L.orc_dt_limit.argtypes, L.orc_dt_limit.restype = [P, dp], C.c_int
            _lib = L
    return _lib


def params(d: dict) -> OrcParams:
    p = OrcParams()
    for name, _ in OrcParams._fields_:
        setattr(p, name, d[name])
    return p


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---- pointwise functions (for pins) -------------------------------------
def p_fn(x): return lib().orc_p(float(x))
def dp_fn(x): return lib().orc_dp(float(x))
def h_fn(x): return lib().orc_h(float(x))
def g_fn(x): return lib().orc_g(float(x))
def dg_fn(x): return lib().orc_dg(float(x))
def f_fn(pd, phi, c): return lib().orc_f(C.byref(params(pd)), float(phi), float(c))
def mobility(pd, phi, c): return lib().orc_mobility(C.byref(params(pd)), float(phi), float(c))


def dt_limit(pd: dict) -> dict:
    out = np.zeros(4)
    lib().orc_dt_limit(C.byref(params(pd)), out)
    return dict(dt_lim=out[0], dt_c=out[1], dt_phi=out[2], dt_rho=out[3])


def chem_pot(pd, phi, c):
    phi, c = _f64(phi), _f64(c)
    ny, nx = phi.shape
    mc, mf = np.empty_like(phi), np.empty_like(phi)
    rc = lib().orc_chem_pot(C.byref(params(pd)), nx, ny, phi, c, mc, mf)
    assert rc == 0
    return mc, mf


def rhs(pd, phi, c, rho):
    phi, c, rho = _f64(phi), _f64(c), _f64(rho)
    ny, nx = phi.shape
    Rf, Rc, Rr = np.empty_like(phi), np.empty_like(phi), np.empty_like(phi)
    rc = lib().orc_rhs(C.byref(params(pd)), nx, ny, phi, c, rho, Rf, Rc, Rr)
    assert rc == 0
    return Rf, Rc, Rr


def step(pd, phi, c, rho, nsteps: int):
    """Advance copies of (phi, c, rho) by nsteps explicit midpoint steps; returns FP64 arrays."""
    phi, c, rho = _f64(phi).copy(), _f64(c).copy(), _f64(rho).copy()
    ny, nx = phi.shape
    rc = lib().orc_step(C.byref(params(pd)), nx, ny, phi, c, rho, int(nsteps))
    assert rc == 0
    return phi, c, rho


def free_energy(pd, phi, c) -> float:
    phi, c = _f64(phi), _f64(c)
    ny, nx = phi.shape
    return lib().orc_free_energy(C.byref(params(pd)), nx, ny, phi, c)


def diag(pd, phi, c, rho) -> np.ndarray:
    """[dx^2 sum c, dx^2 sum phi, dx^2 sum rho, F_h]"""
    phi, c, rho = _f64(phi), _f64(c), _f64(rho)
    ny, nx = phi.shape
    out = np.zeros(4)
    lib().orc_diag(C.byref(params(pd)), nx, ny, phi, c, rho, out)
    return out


def with_dt(pd: dict, frac: float = 0.5) -> dict:
    """Copy of pd with dt = frac x the oracle's stability limit."""
    q = dict(pd)
    q["dt"] = frac * dt_limit(pd)["dt_lim"]
    return q
