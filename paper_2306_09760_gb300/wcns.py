"""Python binding of libwcns (the C ABI in include/wcns.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Functions keep the C names (`wcns_init`, `wcns_rhs`, `wcns_step`, ...).
Device buffers are passed as torch CUDA tensors (or raw integer pointers); PyTorch
supplies device memory and streams, nothing else.

The binding refuses to work without the compiled library: there is no fallback.
Build it with `python -m paper_2306_09760_gb300.build` (or `__graft_entry__.build()`).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwcns.so")

WCNS_OK, WCNS_ERR_ARG, WCNS_ERR_CUDA, WCNS_ERR_NONPHYSICAL, WCNS_ERR_TIMEOUT, WCNS_ERR_UNSUPPORTED, \
    WCNS_ERR_NOMEM = range(7)
WCNS_F64, WCNS_F32 = 0, 1
WCNS_BC_PERIODIC, WCNS_BC_TRANSMISSIVE = 0, 1
WCNS_ADVECTION, WCNS_EULER = 0, 1
WEIGHTS = {"JS": 0, "Z": 1, "FE": 2, "PFE": 3, "M": 4}
FLUXES = {"LLF": 0, "ROE": 1, "HLLC": 2, "LLF_FROZEN": 3}
WCNS_REDUCE_SUM, WCNS_REDUCE_L1, WCNS_REDUCE_LINF, WCNS_REDUCE_MAXWAVE = range(4)
WCNS_RK3, WCNS_RK4 = 0, 1
INTEGRATORS = {"RK3": 0, "RK4": 1}
FAMILIES = {"WCNS": 0, "WENO": 1}


class WcnsError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {wcns_status_string(status)} (status {status})")


class wcns_grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("nvar", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("pitch", ctypes.c_int64), ("lo", ctypes.c_double * 2), ("hi", ctypes.c_double * 2),
                ("bc", ctypes.c_int32 * 2)]


class wcns_params(ctypes.Structure):
    _fields_ = [("system", ctypes.c_int32), ("weights", ctypes.c_int32), ("flux", ctypes.c_int32),
                ("characteristic", ctypes.c_int32), ("z_p", ctypes.c_int32), ("renorm", ctypes.c_int32),
                ("integrator", ctypes.c_int32), ("family", ctypes.c_int32), ("adv_speed", ctypes.c_double * 2),
                ("gamma", ctypes.c_double),
                ("eps", ctypes.c_double), ("xi", ctypes.c_double), ("kappa", ctypes.c_double),
                ("cv", ctypes.c_double), ("cfl", ctypes.c_double), ("alpha", ctypes.c_double * 2),
                ("harten", ctypes.c_double)]


class wcns_faces(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32 * 4), ("reserved", ctypes.c_int32 * 4),
                ("state_a", ctypes.c_double * 4), ("state_b", ctypes.c_double * 4),
                ("wall_x", ctypes.c_double), ("shock_x0", ctypes.c_double),
                ("shock_dxdy", ctypes.c_double), ("shock_speed", ctypes.c_double)]


_lib = None


def load():
    """Loads libwcns.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libwcns.so is not built ({LIB_PATH}); run `python -m paper_2306_09760_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    st = ctypes.c_int
    sig = {
        "wcns_default_params": (st, [ctypes.c_int32, ctypes.c_int32, P(wcns_params)]),
        "wcns_init": (st, [P(wcns_grid), P(wcns_params), vp, P(vp)]),
        "wcns_rhs": (st, [vp, vp, vp]),
        "wcns_step": (st, [vp, vp, ctypes.c_double, ctypes.c_int32, ctypes.c_double]),
        "wcns_step_host": (st, [vp, vp, ctypes.c_double, ctypes.c_int32, ctypes.c_double]),
        "wcns_set_time": (st, [vp, ctypes.c_double]),
        "wcns_get_time": (st, [vp, P(ctypes.c_double), P(ctypes.c_int64)]),
        "wcns_reduce": (st, [vp, vp, vp, ctypes.c_int32, P(ctypes.c_double)]),
        "wcns_adjoint_step": (st, [vp, vp, ctypes.c_double, vp, vp]),
        "wcns_adjoint_step_stages": (st, [vp, vp, vp, vp, ctypes.c_double, vp, vp]),
        "wcns_step_stages": (st, [vp, vp, ctypes.c_double, vp, vp]),
        "wcns_weight_hist": (st, [vp, vp, ctypes.c_int32, vp]),
        "wcns_set_faces": (st, [vp, vp]),
        "wcns_set_stage_form": (st, [vp, ctypes.c_int32]),
        "wcns_selftest_waits": (st, [vp, P(ctypes.c_int32)]),
        "wcns_reduce_noalloc": (st, [P(wcns_grid), vp, vp, ctypes.c_int32, vp, vp]),
        "wcns_reciprocal_f64": (st, [vp, vp, ctypes.c_int64, vp]),
        "wcns_sync_status": (st, [vp, P(ctypes.c_int64)]),
        "wcns_status_string": (ctypes.c_char_p, [st]),
        "wcns_profile_enable": (st, [vp, ctypes.c_int32]),
        "wcns_profile_read": (st, [vp, ctypes.c_int32, ctypes.c_char_p, P(ctypes.c_int64), P(ctypes.c_double),
                                   P(ctypes.c_int32)]),
        "wcns_destroy": (None, [vp]),
        "wcns_batch_init": (st, [P(ctypes.c_int64), P(ctypes.c_int64), ctypes.c_int32, ctypes.c_int64,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_int32, P(wcns_params), ctypes.c_int32,
                                 ctypes.c_int32, vp, P(vp)]),
        "wcns_batch_step": (st, [vp, vp, ctypes.c_int32, ctypes.c_double]),
        "wcns_batch_config": (st, [vp, P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32)]),
        "wcns_batch_times": (st, [vp, P(ctypes.c_double)]),
        "wcns_batch_sync_status": (st, [vp, P(ctypes.c_int64)]),
        "wcns_batch_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _check(status: int, where: str):
    if status != WCNS_OK:
        raise WcnsError(status, where)


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------------------
# C-ABI functions (same names)
# ---------------------------------------------------------------------------
def wcns_status_string(s: int) -> str:
    return load().wcns_status_string(int(s)).decode()


def wcns_default_params(system: int, dtype: int) -> wcns_params:
    p = wcns_params()
    _check(load().wcns_default_params(system, dtype, ctypes.byref(p)), "wcns_default_params")
    return p


def wcns_init(grid: wcns_grid, params: wcns_params, stream=None) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(load().wcns_init(ctypes.byref(grid), ctypes.byref(params), _stream_handle(stream), ctypes.byref(ctx)),
           "wcns_init")
    return ctx


def wcns_rhs(ctx, u, dudt):
    _check(load().wcns_rhs(ctx, _ptr(u), _ptr(dudt)), "wcns_rhs")


def wcns_step(ctx, u, dt: float, nsteps: int, t_end: float = 0.0):
    _check(load().wcns_step(ctx, _ptr(u), float(dt), int(nsteps), float(t_end)), "wcns_step")


def wcns_step_host(ctx, u_host, dt: float, nsteps: int, t_end: float = 0.0):
    _check(load().wcns_step_host(ctx, _ptr(u_host), float(dt), int(nsteps), float(t_end)), "wcns_step_host")


def wcns_set_time(ctx, t: float):
    _check(load().wcns_set_time(ctx, float(t)), "wcns_set_time")


def wcns_get_time(ctx):
    t = ctypes.c_double()
    n = ctypes.c_int64()
    _check(load().wcns_get_time(ctx, ctypes.byref(t), ctypes.byref(n)), "wcns_get_time")
    return t.value, n.value


def wcns_reduce(ctx, a, b, what: int, nout: int) -> np.ndarray:
    out = np.zeros(max(nout, 4))
    _check(load().wcns_reduce(ctx, _ptr(a), _ptr(b), int(what), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
           "wcns_reduce")
    return out[:nout]


def wcns_reduce_noalloc(grid: wcns_grid, a, b, what: int, out_dev, stream=None):
    """Context-free, allocation-free reduction; `out_dev` is a device buffer of nvar doubles."""
    _check(load().wcns_reduce_noalloc(ctypes.byref(grid), _ptr(a), _ptr(b), int(what), _stream_handle(stream),
                                      _ptr(out_dev)), "wcns_reduce_noalloc")


def wcns_reciprocal_f64(x, out, stream=None):
    """The library's double-precision device reciprocal applied to a device tensor."""
    _check(load().wcns_reciprocal_f64(_ptr(x), _ptr(out), int(x.numel()), _stream_handle(stream)),
           "wcns_reciprocal_f64")


def wcns_weight_hist(ctx, u, nbins: int, hist):
    """App. A weight statistics of one L(u), added into the device uint64 tensor `hist`
    (6 * nbins counters, layout [kind][k][bin])."""
    _check(load().wcns_weight_hist(ctx, _ptr(u), int(nbins), _ptr(hist)), "wcns_weight_hist")


def wcns_set_faces(ctx, faces=None):
    """Boundary faces from a dict {"types": 4 ints, "state_a", "state_b", "wall_x",
    "shock": (x0, dxdy, speed)} (the layout of inputs' Problem.extra["faces"]); None resets."""
    if faces is None:
        _check(load().wcns_set_faces(ctx, None), "wcns_set_faces")
        return
    f = wcns_faces()
    for k in range(4):
        f.type[k] = int(faces["types"][k])
        f.state_a[k] = float(faces.get("state_a", (0.0,) * 4)[k])
        f.state_b[k] = float(faces.get("state_b", (0.0,) * 4)[k])
    f.wall_x = float(faces.get("wall_x", 0.0))
    f.shock_x0, f.shock_dxdy, f.shock_speed = (float(v) for v in faces.get("shock", (0.0, 0.0, 0.0)))
    _check(load().wcns_set_faces(ctx, ctypes.byref(f)), "wcns_set_faces")


def wcns_adjoint_step(ctx, u_n, dt: float, lam_np1, lam_n):
    _check(load().wcns_adjoint_step(ctx, _ptr(u_n), float(dt), _ptr(lam_np1), _ptr(lam_n)), "wcns_adjoint_step")


def wcns_adjoint_step_stages(ctx, u_n, u1, u2, dt: float, lam_np1, lam_n):
    _check(load().wcns_adjoint_step_stages(ctx, _ptr(u_n), _ptr(u1), _ptr(u2), float(dt), _ptr(lam_np1),
                                           _ptr(lam_n)), "wcns_adjoint_step_stages")


def wcns_step_stages(ctx, u, dt: float, u1_out, u2_out):
    _check(load().wcns_step_stages(ctx, _ptr(u), float(dt), _ptr(u1_out), _ptr(u2_out)), "wcns_step_stages")


def wcns_sync_status(ctx):
    """Returns (status, nonphysical_interfaces) without raising."""
    n = ctypes.c_int64()
    s = load().wcns_sync_status(ctx, ctypes.byref(n))
    return s, n.value


def wcns_selftest_waits(ctx):
    """[counter wait gave up, mbarrier wait gave up] (both should be 1)."""
    out = (ctypes.c_int32 * 2)()
    _check(load().wcns_selftest_waits(ctx, out), "wcns_selftest_waits")
    return [int(out[0]), int(out[1])]


def wcns_set_stage_form(ctx, banded: bool):
    _check(load().wcns_set_stage_form(ctx, int(bool(banded))), "wcns_set_stage_form")


def wcns_profile_enable(ctx, on: bool):
    _check(load().wcns_profile_enable(ctx, int(bool(on))), "wcns_profile_enable")


def wcns_profile_read(ctx) -> dict:
    """{kernel kind: (launches, total ms)} since the last read."""
    n = 16
    names = ctypes.create_string_buffer(48 * n)
    launches = (ctypes.c_int64 * n)()
    ms = (ctypes.c_double * n)()
    cnt = ctypes.c_int32()
    _check(load().wcns_profile_read(ctx, n, names, launches, ms, ctypes.byref(cnt)), "wcns_profile_read")
    out = {}
    for k in range(cnt.value):
        name = names.raw[48 * k: 48 * (k + 1)].split(b"\0", 1)[0].decode()
        out[name] = (int(launches[k]), float(ms[k]))
    return out


def wcns_destroy(ctx):
    if ctx:
        load().wcns_destroy(ctx)


def wcns_batch_init(offsets, sizes, total, lo, hi, bc, params, dtype, tile=0, stream=None):
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    sizes = np.ascontiguousarray(sizes, dtype=np.int64)
    b = ctypes.c_void_p()
    P64 = ctypes.POINTER(ctypes.c_int64)
    _check(load().wcns_batch_init(offsets.ctypes.data_as(P64), sizes.ctypes.data_as(P64), len(sizes), int(total),
                                  float(lo), float(hi), int(bc), ctypes.byref(params), int(dtype), int(tile),
                                  _stream_handle(stream), ctypes.byref(b)), "wcns_batch_init")
    return b


def wcns_batch_step(b, u, nsteps: int, t_end: float = 0.0):
    _check(load().wcns_batch_step(b, _ptr(u), int(nsteps), float(t_end)), "wcns_batch_step")


def wcns_batch_config(b):
    t, k, n = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().wcns_batch_config(b, ctypes.byref(t), ctypes.byref(k), ctypes.byref(n)), "wcns_batch_config")
    return t.value, k.value, n.value


def wcns_batch_times(b, nprob: int) -> np.ndarray:
    out = np.zeros(nprob)
    _check(load().wcns_batch_times(b, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "wcns_batch_times")
    return out


def wcns_batch_sync_status(b):
    n = ctypes.c_int64()
    s = load().wcns_batch_sync_status(b, ctypes.byref(n))
    return s, n.value


def wcns_batch_destroy(b):
    if b:
        load().wcns_batch_destroy(b)


# ---------------------------------------------------------------------------
# Convenience layer
# ---------------------------------------------------------------------------
def make_params(system: int, dtype: int, **kw) -> wcns_params:
    """Library defaults (wcns_default_params) overridden by keyword arguments with the
    same meaning as the struct fields; weights/flux accept names ("FE", "HLLC", ...)."""
    p = wcns_default_params(system, dtype)
    for k, v in kw.items():
        if k == "weights":
            p.weights = WEIGHTS[v] if isinstance(v, str) else int(v)
        elif k == "flux":
            p.flux = FLUXES[v] if isinstance(v, str) else int(v)
        elif k in ("zp", "z_p"):
            p.z_p = int(v)
        elif k in ("characteristic", "renorm"):
            setattr(p, k, int(bool(v)))
        elif k == "integrator":
            p.integrator = INTEGRATORS[v] if isinstance(v, str) else int(v)
        elif k == "family":
            p.family = FAMILIES[v] if isinstance(v, str) else int(v)
        elif k in ("alpha", "adv_speed"):
            arr = getattr(p, k)
            arr[0], arr[1] = float(v[0]), float(v[1])
        elif k in ("gamma", "eps", "xi", "kappa", "cv", "cfl", "harten"):
            setattr(p, k, float(v))
        else:
            raise KeyError(k)
    return p


def padded_pitch(nx: int) -> int:
    return (nx + 31) // 32 * 32


class Solver:
    """One grid on the GPU: owns a context and a padded state tensor [nvar, ny, pitch]."""

    def __init__(self, problem, dtype: str = "f64", stream=None, **params):
        import torch
        self.torch = torch
        self.problem = problem
        self.dtype_code = WCNS_F64 if dtype == "f64" else WCNS_F32
        self.tdtype = torch.float64 if dtype == "f64" else torch.float32
        g = wcns_grid()
        g.ndim, g.nvar, g.dtype = problem.ndim, problem.nvar, self.dtype_code
        g.nx, g.ny = problem.nx, problem.ny
        g.pitch = padded_pitch(problem.nx)
        g.lo[0], g.lo[1] = problem.lo
        g.hi[0], g.hi[1] = problem.hi
        g.bc[0], g.bc[1] = problem.bc
        self.grid = g
        kw = dict(params)
        if problem.system == WCNS_ADVECTION:
            kw.setdefault("adv_speed", problem.adv_speed)
        kw.setdefault("gamma", problem.gamma)
        self.params = make_params(problem.system, self.dtype_code, **kw)
        self.stream = stream
        self.ctx = wcns_init(g, self.params, stream)
        faces = problem.extra.get("faces") if problem.extra else None
        if faces:
            wcns_set_faces(self.ctx, faces)
        self.u = self.alloc()
        self.set_state(problem.u0)

    def alloc(self):
        g = self.grid
        t = self.torch.zeros((g.nvar, g.ny, g.pitch), dtype=self.tdtype, device="cuda")
        return t

    def set_state(self, u_np, dst=None):
        dst = self.u if dst is None else dst
        g = self.grid
        host = self.torch.as_tensor(np.ascontiguousarray(u_np).reshape(g.nvar, g.ny, g.nx))
        dst[:, :, : g.nx].copy_(host.to(self.tdtype))
        dst[:, :, g.nx:].zero_()
        return dst

    def view(self, t=None):
        t = self.u if t is None else t
        return t[:, :, : self.grid.nx]

    def numpy(self, t=None):
        self.torch.cuda.synchronize()
        return self.view(t).double().cpu().numpy()

    def rhs(self, u=None):
        out = self.alloc()
        wcns_rhs(self.ctx, self.u if u is None else u, out)
        return out

    def step(self, dt=0.0, nsteps=1, t_end=0.0):
        wcns_step(self.ctx, self.u, dt, nsteps, t_end)

    def run_to(self, t_end, chunk=64, max_steps=10 ** 7):
        steps = 0
        while steps < max_steps:
            self.step(0.0, chunk, t_end)
            steps += chunk
            t, _ = wcns_get_time(self.ctx)
            if t >= t_end:
                break
        return wcns_get_time(self.ctx)

    def time(self):
        return wcns_get_time(self.ctx)

    def status(self):
        return wcns_sync_status(self.ctx)

    def reduce(self, what, a=None, b=None):
        n = self.grid.ndim if what == WCNS_REDUCE_MAXWAVE else self.grid.nvar
        return wcns_reduce(self.ctx, self.u if a is None else a, b, what, n)

    def close(self):
        if self.ctx:
            wcns_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
