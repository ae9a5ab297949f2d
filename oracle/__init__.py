"""FP64 CPU oracle for the WCNS-FE hot path -- TEST INFRASTRUCTURE ONLY.

Only the tests, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg may
import this package.  The product path (the CUDA library and its binding) never
does, and shares no code with it.  See `wcns_oracle.cpp` for the paper passages each
function follows.

Parity status: every function is pinned by `tests/test_oracle_*.py` against values
the paper prints (Table 1 and Table B.1 control values), closed forms (the linear scheme's Fourier
symbol, polynomial exactness, Eq. 18 truncation coefficients, the exact Riemann
solution, the JS, M and Z weights of Eq. 11-15 in exact rational arithmetic, the CFL
step of uniform states and of the Sod tube), invariants (conservation, symmetry) and
central finite differences.  The weight statistics (`weight_hist`) are pinned by a
brute-force enumeration of one L(u)'s one-sided interpolations with the Z weights of
Eq. 14-15 in exact fractions and the Table 1 staircase, and by the sample counts that
Eq. 3 and App. B fix; the absolute shares of Tables A.1-A.4 are not reproduced, since
they depend on solver settings the paper does not state.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wcns_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle_wcns.so")

WEIGHTS = {"JS": 0, "Z": 1, "FE": 2, "PFE": 3, "M": 4}
FLUXES = {"LLF": 0, "ROE": 1, "HLLC": 2, "LLF_FROZEN": 3}
FAMILIES = {"WCNS": 0, "WENO": 1}


class OracleCfg(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int32), ("nvar", ctypes.c_int32),
        ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
        ("hx", ctypes.c_double), ("hy", ctypes.c_double),
        ("bcx", ctypes.c_int32), ("bcy", ctypes.c_int32),
        ("system", ctypes.c_int32), ("weights", ctypes.c_int32),
        ("flux", ctypes.c_int32), ("characteristic", ctypes.c_int32),
        ("zp", ctypes.c_int32), ("renorm", ctypes.c_int32),
        ("ax", ctypes.c_double), ("ay", ctypes.c_double),
        ("gamma", ctypes.c_double), ("eps", ctypes.c_double),
        ("xi", ctypes.c_double), ("kappa", ctypes.c_double),
        ("cv", ctypes.c_double),
        ("alpha_x", ctypes.c_double), ("alpha_y", ctypes.c_double),
        ("harten", ctypes.c_double),
        ("family", ctypes.c_int32), ("pad_", ctypes.c_int32),
        ("face", ctypes.c_int32 * 4),
        ("state_a", ctypes.c_double * 4), ("state_b", ctypes.c_double * 4),
        ("wall_x", ctypes.c_double), ("shock_x0", ctypes.c_double),
        ("shock_dxdy", ctypes.c_double), ("shock_speed", ctypes.c_double),
        ("lo_x", ctypes.c_double), ("lo_y", ctypes.c_double),
        ("time", ctypes.c_double),
    ]


DEFAULTS = dict(weights="FE", flux="HLLC", characteristic=True, zp=1, renorm=True,
                eps=1e-40, xi=1e6, kappa=0.5, cv=1e-3, alpha=(0.0, 0.0), harten=0.1, cfl=0.5,
                family="WCNS")


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (OpenMP, no FP contraction).  Returns the library path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-std=c++17", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.POINTER
        dp = P(ctypes.c_double)
        cp = P(OracleCfg)
        L.oracle_fe_map.restype = ctypes.c_double
        L.oracle_fe_map.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.oracle_fe_map_family.restype = ctypes.c_double
        L.oracle_fe_map_family.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double]
        L.oracle_fe_map_deriv.restype = ctypes.c_double
        L.oracle_fe_map_deriv.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.oracle_m_map.restype = ctypes.c_double
        L.oracle_m_map.argtypes = [ctypes.c_double, ctypes.c_double]
        L.oracle_interp.restype = ctypes.c_double
        L.oracle_interp.argtypes = [cp, dp, dp, dp, P(ctypes.c_int)]
        L.oracle_eigenvectors.restype = None
        L.oracle_eigenvectors.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, dp, dp]
        L.oracle_interface_flux.restype = ctypes.c_int
        L.oracle_interface_flux.argtypes = [cp, dp, dp]
        L.oracle_riemann.restype = None
        L.oracle_riemann.argtypes = [cp, dp, dp, dp]
        L.oracle_rhs.restype = ctypes.c_longlong
        L.oracle_rhs.argtypes = [cp, dp, dp]
        L.oracle_weight_hist.restype = ctypes.c_longlong
        L.oracle_weight_hist.argtypes = [cp, dp, P(ctypes.c_longlong), ctypes.c_int]
        L.oracle_rhs_cells.restype = None
        L.oracle_rhs_cells.argtypes = [cp, dp, ctypes.c_int64, P(ctypes.c_int64), dp]
        L.oracle_max_wave.restype = None
        L.oracle_max_wave.argtypes = [cp, dp, dp, dp]
        L.oracle_step.restype = ctypes.c_int
        L.oracle_step.argtypes = [cp, dp, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                  dp, P(ctypes.c_longlong)]
        L.oracle_step_rk4.restype = ctypes.c_int
        L.oracle_step_rk4.argtypes = [cp, dp, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
        L.oracle_rhs_jvp.restype = None
        L.oracle_rhs_jvp.argtypes = [cp, dp, dp, dp, dp]
        L.oracle_step_jvp.restype = None
        L.oracle_step_jvp.argtypes = [cp, dp, dp, ctypes.c_double, ctypes.c_int]
        L.oracle_count_rhs_flops.restype = ctypes.c_double
        L.oracle_count_rhs_flops.argtypes = [cp, dp]
        L.oracle_set_threads.restype = None
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_max_threads.restype = ctypes.c_int
        L.oracle_max_threads.argtypes = []
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_cfg(problem=None, **params) -> OracleCfg:
    """Oracle configuration from an `inputs.Problem` and scheme parameters."""
    p = dict(DEFAULTS)
    p.update(params)
    c = OracleCfg()
    if problem is not None:
        c.ndim, c.nvar = problem.ndim, problem.nvar
        c.nx, c.ny = problem.nx, problem.ny
        hx, hy = problem.h
        c.hx, c.hy = hx, hy
        c.bcx, c.bcy = problem.bc
        c.system = problem.system
        c.ax, c.ay = problem.adv_speed
        c.gamma = problem.gamma
        c.lo_x, c.lo_y = problem.lo
        faces = problem.extra.get("faces") if problem.extra else None
        if faces:
            for f in range(4):
                c.face[f] = int(faces["types"][f])
            for k in range(4):
                c.state_a[k] = faces.get("state_a", (0.0,) * 4)[k]
                c.state_b[k] = faces.get("state_b", (0.0,) * 4)[k]
            c.wall_x = faces.get("wall_x", 0.0)
            c.shock_x0, c.shock_dxdy, c.shock_speed = faces.get("shock", (0.0, 0.0, 0.0))
    else:
        c.ndim, c.nvar, c.nx, c.ny, c.hx, c.hy = 1, 1, 1, 1, 1.0, 1.0
        c.system, c.gamma = 0, 1.4
    c.weights = WEIGHTS[p["weights"]] if isinstance(p["weights"], str) else int(p["weights"])
    c.flux = FLUXES[p["flux"]] if isinstance(p["flux"], str) else int(p["flux"])
    c.characteristic = int(bool(p["characteristic"]))
    c.zp, c.renorm = int(p["zp"]), int(bool(p["renorm"]))
    c.eps, c.xi, c.kappa, c.cv = p["eps"], p["xi"], p["kappa"], p["cv"]
    c.alpha_x, c.alpha_y = p["alpha"]
    c.harten = p["harten"]
    c.family = FAMILIES[p["family"]] if isinstance(p["family"], str) else int(p["family"])
    c.time = float(params.get("time", 0.0))
    if "gamma" in params:
        c.gamma = params["gamma"]
    return c


def set_threads(n: int):
    lib().oracle_set_threads(int(n))


def max_threads() -> int:
    return lib().oracle_max_threads()


def fe_map(i: int, w: float, xi: float = 1e6, kappa: float = 0.5) -> float:
    """Eq. 20 (with phi of Eq. 21) for weight index i."""
    return lib().oracle_fe_map(i, w, xi, kappa)


def fe_map_weno(i: int, w: float, xi: float = 1e6, kappa: float = 0.5) -> float:
    """Eq. 20 with the control rows of App. B, Table B.2 (FE-WENO family)."""
    return lib().oracle_fe_map_family(1, i, w, xi, kappa)


def fe_map_deriv(i: int, w: float, xi: float = 1e6, kappa: float = 0.5) -> float:
    return lib().oracle_fe_map_deriv(i, w, xi, kappa)


def m_map(w: float, d: float) -> float:
    """Eq. 13 (Henrick's mapping) at w for ideal weight d."""
    return lib().oracle_m_map(w, d)


def interp(v5, **params):
    """One-sided midpoint interpolation of (u_{i-2}..u_{i+2}).  Returns (value, w_base, w_final, mapped)."""
    c = make_cfg(None, **params)
    v = np.ascontiguousarray(v5, dtype=np.float64)
    wz = np.zeros(3); wf = np.zeros(3); m = ctypes.c_int(0)
    r = lib().oracle_interp(ctypes.byref(c), _dp(v), _dp(wz), _dp(wf), ctypes.byref(m))
    return r, wz, wf, m.value


def eigenvectors(nvar, gamma, u, v, H, c):
    Rm = np.zeros(16); Lm = np.zeros(16)
    lib().oracle_eigenvectors(nvar, gamma, u, v, H, c, _dp(Rm), _dp(Lm))
    return Rm.reshape(4, 4)[:nvar, :nvar].copy(), Lm.reshape(4, 4)[:nvar, :nvar].copy()


def riemann(UL, UR, nvar, **params):
    c = make_cfg(None, **params)
    c.nvar = nvar
    c.system = 1
    a = np.ascontiguousarray(UL, dtype=np.float64); b = np.ascontiguousarray(UR, dtype=np.float64)
    F = np.zeros(nvar)
    lib().oracle_riemann(ctypes.byref(c), _dp(a), _dp(b), _dp(F))
    return F


def interface_flux(S, nvar, system=1, ax=1.0, **params):
    """Midpoint flux between cells 2 and 3 of six stencil states S[6, nvar] (x normal).
    Returns (F, fell_back)."""
    c = make_cfg(None, **params)
    c.nvar, c.system, c.ax = nvar, system, ax
    S = np.ascontiguousarray(S, dtype=np.float64)
    F = np.zeros(nvar)
    fb = lib().oracle_interface_flux(ctypes.byref(c), _dp(S), _dp(F))
    return F, bool(fb)


def rhs(problem, u=None, **params):
    """L(u) on the whole grid; returns (dudt [nvar, ny, nx], nonphysical_count)."""
    c = make_cfg(problem, **params)
    u = np.ascontiguousarray(problem.u0 if u is None else u, dtype=np.float64)
    out = np.zeros_like(u)
    n = lib().oracle_rhs(ctypes.byref(c), _dp(u), _dp(out))
    return out, n


def rhs_cells(problem, u, cells, **params):
    """L(u) at flattened cell indices j*nx + i; returns [ncells, nvar]."""
    c = make_cfg(problem, **params)
    u = np.ascontiguousarray(u, dtype=np.float64)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    out = np.zeros((len(cells), problem.nvar))
    lib().oracle_rhs_cells(ctypes.byref(c), _dp(u), len(cells),
                           cells.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(out))
    return out


def max_wave(problem, u=None, **params):
    c = make_cfg(problem, **params)
    u = np.ascontiguousarray(problem.u0 if u is None else u, dtype=np.float64)
    wx = ctypes.c_double(); wy = ctypes.c_double()
    lib().oracle_max_wave(ctypes.byref(c), _dp(u), ctypes.byref(wx), ctypes.byref(wy))
    return wx.value, wy.value


def step(problem, u=None, dt=0.0, nsteps=1, t_end=0.0, t0=0.0, cfl=None, rk4=False, **params):
    """TVD-RK3 steps (RK4 of Eq. 16 if rk4).  dt <= 0 selects the CFL step; t_end > 0 clips.
    Returns (u, t, steps_taken, nonphysical_count)."""
    c = make_cfg(problem, **params)
    u = np.array(problem.u0 if u is None else u, dtype=np.float64, order="C", copy=True)
    cfl = DEFAULTS["cfl"] if cfl is None else cfl
    t = ctypes.c_double(t0)
    nonph = ctypes.c_longlong(0)
    if rk4:
        taken = lib().oracle_step_rk4(ctypes.byref(c), _dp(u), dt, nsteps, cfl, t_end, ctypes.byref(t))
    else:
        taken = lib().oracle_step(ctypes.byref(c), _dp(u), dt, nsteps, cfl, t_end, ctypes.byref(t),
                                  ctypes.byref(nonph))
    return u, t.value, taken, nonph.value


def run_to(problem, t_end, u=None, max_steps=10 ** 7, **params):
    """Advance with CFL steps until t_end."""
    return step(problem, u=u, dt=0.0, nsteps=max_steps, t_end=t_end, **params)


def rhs_jvp(problem, u, du, **params):
    c = make_cfg(problem, **params)
    u = np.ascontiguousarray(u, dtype=np.float64); du = np.ascontiguousarray(du, dtype=np.float64)
    L = np.zeros_like(u); dL = np.zeros_like(u)
    lib().oracle_rhs_jvp(ctypes.byref(c), _dp(u), _dp(du), _dp(L), _dp(dL))
    return L, dL


def step_jvp(problem, u, du, dt, nsteps, **params):
    """Fixed-dt TVD-RK3 steps carrying a tangent; returns (u_T, du_T)."""
    c = make_cfg(problem, **params)
    u = np.array(u, dtype=np.float64, order="C", copy=True)
    du = np.array(du, dtype=np.float64, order="C", copy=True)
    lib().oracle_step_jvp(ctypes.byref(c), _dp(u), _dp(du), dt, nsteps)
    return u, du


def count_rhs_flops(problem, u=None, **params) -> float:
    c = make_cfg(problem, **params)
    u = np.ascontiguousarray(problem.u0 if u is None else u, dtype=np.float64)
    return lib().oracle_count_rhs_flops(ctypes.byref(c), _dp(u))


def weight_hist(problem, u=None, nbins=10000, **params):
    """Histogram [2, 3, nbins] of (base, final) weights over all one-sided interpolations."""
    c = make_cfg(problem, **params)
    u = np.ascontiguousarray(problem.u0 if u is None else u, dtype=np.float64)
    h = np.zeros((2, 3, nbins), dtype=np.int64)
    n = lib().oracle_weight_hist(ctypes.byref(c), _dp(u), h.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                                 nbins)
    return h, n
