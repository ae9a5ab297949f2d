"""Seeded synthetic inputs for the WCNS-FE solvers.

This module generates initial data only.  It holds none of the scheme's arithmetic:
no interpolation, weights, fluxes or time stepping.  Both the CUDA path and the CPU
oracle take their inputs from here, so the two sides see identical arrays.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), mapped to doubles in [0, 1) by taking
the top 53 bits.  Every generator is a pure function of its seed.

Layout of every state array: float64, shape [nvar, ny, nx], C-contiguous, conservative
variables (rho, rho*u, [rho*v,] E) for the Euler equations.

Workloads (paper section in brackets):
  * advection_sine   -- u_t + u_x = 0 on periodic [-1, 1], u0 = sin(pi x)   [Sec. 4.1 stand-in]
  * sod, lax         -- shock tubes on [0, 1]                                [Eq. 33, 34]
  * shu_osher        -- Mach-3 shock into rho = 1 + 0.2 sin(5x) on [-5, 5]   [Eq. 35]
  * titarev_toro     -- shock into rho = 1 + 0.1 sin(20 pi x)                [Eq. 36]
  * riemann2d        -- four-quadrant 2D Riemann data split at x = y = 0.8   [Eq. 38]
  * batched_1d       -- many independent uneven-size 1D Euler problems
  * vortex           -- isentropic vortex on periodic [0, 10]^2 with seeded density noise
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_M64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator; `uniform()` returns doubles in [0, 1)."""

    def __init__(self, seed: int):
        self.state = seed & _M64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / 9007199254740992.0))

    def integers(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive)."""
        return lo + int(self.uniform() * (hi - lo + 1))

    def uniform_array(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        """n uniforms, vectorised; identical to n calls of uniform()."""
        k = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.state) + k * np.uint64(0x9E3779B97F4A7C15)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        self.state = (self.state + n * 0x9E3779B97F4A7C15) & _M64
        return lo + (hi - lo) * ((z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0))


@dataclass
class Problem:
    """A grid, boundary conditions and an initial state."""

    name: str
    ndim: int
    nvar: int
    nx: int
    ny: int
    lo: tuple
    hi: tuple
    bc: tuple            # per direction: 0 periodic, 1 transmissive
    u0: np.ndarray       # [nvar, ny, nx] float64
    system: int          # 0 scalar advection, 1 Euler
    t_end: float = 0.0
    adv_speed: tuple = (1.0, 0.0)
    gamma: float = 1.4
    extra: dict = field(default_factory=dict)

    @property
    def h(self):
        return ((self.hi[0] - self.lo[0]) / self.nx,
                (self.hi[1] - self.lo[1]) / self.ny if self.ndim == 2 else 1.0)


def prim_to_cons(rho, u, v, p, gamma=1.4, ndim=1):
    """Primitive (rho, u, [v,] p) to conservative (rho, rho u, [rho v,] E) variables."""
    rho = np.asarray(rho, dtype=np.float64)
    if ndim == 1:
        E = p / (gamma - 1.0) + 0.5 * rho * u * u
        return np.stack([rho, rho * u, E])
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E])


def cell_centres(lo, hi, n):
    h = (hi - lo) / n
    return lo + (np.arange(n) + 0.5) * h


def advection_sine(n=200):
    """u_t + u_x = 0 on periodic [-1, 1]; nodes x_j = -1 + j h (Sec. 2 grid), u0 = sin(pi x)."""
    h = 2.0 / n
    x = -1.0 + np.arange(n) * h
    u0 = np.sin(np.pi * x)[None, None, :].copy()
    return Problem("advection_sine", 1, 1, n, 1, (-1.0, 0.0), (1.0, 1.0), (0, 0), u0, 0,
                   t_end=2.0, adv_speed=(1.0, 0.0), extra={"x": x})


def _tube(name, n, lo, hi, x0, left, right_fn, t_end, gamma=1.4):
    x = cell_centres(lo, hi, n)
    rho = np.empty(n); u = np.empty(n); p = np.empty(n)
    L = x < x0
    rho[L], u[L], p[L] = left
    rr, ur, pr = right_fn(x[~L])
    rho[~L], u[~L], p[~L] = rr, ur, pr
    u0 = prim_to_cons(rho, u, None, p, gamma, 1)[:, None, :].copy()
    return Problem(name, 1, 3, n, 1, (lo, 0.0), (hi, 1.0), (1, 1), u0, 1, t_end=t_end,
                   gamma=gamma, extra={"x": x})


def sod(n=4096):
    """Sod tube (Eq. 33) rescaled to [0, 1] with the interface at 0.5, t = 0.2."""
    return _tube("sod", n, 0.0, 1.0, 0.5, (1.0, 0.0, 1.0),
                 lambda x: (0.125 + 0 * x, 0 * x, 0.1 + 0 * x), 0.2)


def lax(n=4096):
    """Lax tube (Eq. 34) on [0, 1] with the interface at 0.5, t = 0.15."""
    return _tube("lax", n, 0.0, 1.0, 0.5, (0.445, 0.698, 3.528),
                 lambda x: (0.5 + 0 * x, 0 * x, 0.571 + 0 * x), 0.15)


def shu_osher(n=4096):
    """Shu-Osher (Eq. 35) on [-5, 5]: left state for x < -4, right rho = 1 + 0.2 sin(5x); t = 1.8."""
    return _tube("shu_osher", n, -5.0, 5.0, -4.0, (3.857143, 2.629369, 10.33333),
                 lambda x: (1.0 + 0.2 * np.sin(5.0 * x), 0 * x, 1.0 + 0 * x), 1.8)


def titarev_toro(n=2001):
    """Titarev-Toro (Eq. 36) on [0, 10]: left state for x <= 3.5, right rho = 1 + 0.1 sin(20 pi x); t = 4."""
    return _tube("titarev_toro", n, 0.0, 10.0, 3.5, (1.515695, 0.523346, 1.805),
                 lambda x: (1.0 + 0.1 * np.sin(20.0 * np.pi * x), 0 * x, 1.0 + 0 * x), 4.0)


# Eq. 38 quadrant states (rho, u, v, p): Q1 = x>=0.8,y>=0.8; Q2 = x<0.8,y>=0.8;
# Q3 = x<0.8,y<0.8; Q4 = x>=0.8,y<0.8.
EQ38_STATES = ((1.5, 0.0, 0.0, 1.5), (0.5323, 1.206, 0.0, 0.3),
               (0.138, 1.206, 1.206, 0.029), (0.5323, 0.0, 1.206, 0.3))


def riemann2d_states(seed):
    """Four quadrant states; seed "eq38" gives the paper's states, an int draws them:
    rho ~ U[0.1, 1.5], u, v ~ U[-1, 1], p ~ U[0.03, 1.5]."""
    if seed == "eq38":
        return EQ38_STATES
    g = SplitMix64(int(seed) * 7919 + 17)
    return tuple((g.uniform(0.1, 1.5), g.uniform(-1.0, 1.0), g.uniform(-1.0, 1.0), g.uniform(0.03, 1.5))
                 for _ in range(4))


def riemann2d(n=2048, seed=0, ny=None):
    """2D Euler on [0, 1]^2, transmissive, quadrants split at x = y = 0.8 (Eq. 38 layout)."""
    ny = n if ny is None else ny
    x = cell_centres(0.0, 1.0, n)
    y = cell_centres(0.0, 1.0, ny)
    X, Y = np.meshgrid(x, y)  # [ny, nx]
    st = riemann2d_states(seed)
    q = np.where(X >= 0.8, np.where(Y >= 0.8, 0, 3), np.where(Y >= 0.8, 1, 2))
    prim = np.array(st)  # [4, 4]
    rho, u, v, p = (prim[q, k] for k in range(4))
    u0 = prim_to_cons(rho, u, v, p, 1.4, 2)
    return Problem(f"riemann2d_{seed}", 2, 4, n, ny, (0.0, 0.0), (1.0, 1.0), (1, 1), u0, 1,
                   extra={"states": st})


# Boundary face types (x-lo, x-hi, y-lo, y-hi) of a Problem's extra["faces"]: 0 the
# direction's bc, 1 transmissive, 2 inviscid wall, 3 fixed state A, 4 state A for
# x < wall_x and a wall beyond, 5 moving oblique shock (state A for
# x < x0 + (y + speed t) dxdy, state B beyond).  States are primitive (rho, u, v, p).
FACE_GRID, FACE_TRANSMISSIVE, FACE_WALL, FACE_FIXED, FACE_FIXED_THEN_WALL, FACE_SHOCK = range(6)

DMR_POST = (8.0, 7.145, -4.125, 116.5)
DMR_PRE = (1.4, 0.0, 0.0, 1.0)


def dmr(nx=960, ny=240):
    """Double Mach reflection (Sec. 4.3, Eq. 37): [0, 4] x [0, 1], a Mach 10 shock through
    (1/6, 0) at 60 degrees to the wall; pre-shock state below y = sqrt(3) (x - 1/6),
    post-shock above.  Inflow (post-shock) on the left, outflow on the right, the
    post-shock state under x < 1/6 and an inviscid wall beyond on the bottom, and the
    exact moving shock on the top; t_end = 0.2."""
    x = cell_centres(0.0, 4.0, nx)
    y = cell_centres(0.0, 1.0, ny)
    X, Y = np.meshgrid(x, y)
    pre = Y < np.sqrt(3.0) * (X - 1.0 / 6.0)
    prim = [np.where(pre, a, b) for a, b in zip(DMR_PRE, DMR_POST)]
    u0 = prim_to_cons(prim[0], prim[1], prim[2], prim[3], 1.4, 2)
    faces = {"types": (FACE_FIXED, FACE_TRANSMISSIVE, FACE_FIXED_THEN_WALL, FACE_SHOCK),
             "state_a": DMR_POST, "state_b": DMR_PRE, "wall_x": 1.0 / 6.0,
             "shock": (1.0 / 6.0, 1.0 / np.sqrt(3.0), 20.0)}
    return Problem("dmr", 2, 4, nx, ny, (0.0, 0.0), (4.0, 1.0), (1, 1), u0, 1, t_end=0.2,
                   extra={"faces": faces})


# State ranges of the batched problems.  Drawn as wide as the 2D quadrant states
# (rho from 0.1, p from 0.03, |u| up to 1), a few percent of the problems are
# near-vacuum Riemann problems on which the scheme (which has no positivity limiter)
# produces negative pressure within a few steps; these ranges keep every problem
# physical over the benchmark's steps.
BATCH_RHO = (0.5, 1.5)
BATCH_U = (-0.5, 0.5)
BATCH_P = (0.3, 1.5)


def batched_1d(nprob=4096, seed=0, nmin=64, nmax=8192):
    """Independent 1D Euler problems on [0, 1], transmissive.  Per problem k:
    N_k ~ U{nmin..nmax}; K_k ~ U{1..4} interfaces at sorted U(0, 1) positions;
    piecewise-constant (rho, u, p) with rho ~ U[BATCH_RHO], u ~ U[BATCH_U], p ~ U[BATCH_P];
    density times (1 + 0.1 sin(2 pi m_k x)), m_k ~ U{1..16}.
    Returns (sizes, offsets, u_concat [3, total]) with problem k in columns
    offsets[k] : offsets[k] + sizes[k]."""
    g = SplitMix64(int(seed) * 104729 + 3)
    sizes = np.array([g.integers(nmin, nmax) for _ in range(nprob)], dtype=np.int64)
    offsets = np.zeros(nprob, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)[:-1]
    total = int(sizes.sum())
    u = np.empty((3, total))
    for k in range(nprob):
        n = int(sizes[k])
        x = cell_centres(0.0, 1.0, n)
        K = g.integers(1, 4)
        cuts = np.sort([g.uniform() for _ in range(K)])
        states = [(g.uniform(*BATCH_RHO), g.uniform(*BATCH_U), g.uniform(*BATCH_P)) for _ in range(K + 1)]
        m = g.integers(1, 16)
        seg = np.searchsorted(cuts, x, side="right")
        st = np.array(states)
        rho = st[seg, 0] * (1.0 + 0.1 * np.sin(2.0 * np.pi * m * x))
        u[:, offsets[k]:offsets[k] + n] = prim_to_cons(rho, st[seg, 1], None, st[seg, 2], 1.4, 1)
    return sizes, offsets, u


def vortex_primitive(n, t=0.0, strength=5.0, centre=(5.0, 5.0), mean=(1.0, 1.0), gamma=1.4, L=10.0):
    """Isentropic vortex on periodic [0, L]^2 translated by mean*t (closed form):
    du = -b/(2 pi) (y - yc) e^{(1 - r^2)/2}, dv = b/(2 pi) (x - xc) e^{(1 - r^2)/2},
    T = 1 - (gamma - 1) b^2 / (8 gamma pi^2) e^{1 - r^2}, rho = T^{1/(gamma-1)}, p = rho^gamma."""
    x = cell_centres(0.0, L, n)
    X, Y = np.meshgrid(x, x)
    xc = (centre[0] + mean[0] * t) % L
    yc = (centre[1] + mean[1] * t) % L
    dx = (X - xc + L / 2) % L - L / 2
    dy = (Y - yc + L / 2) % L - L / 2
    r2 = dx * dx + dy * dy
    b = strength
    e = np.exp(0.5 * (1.0 - r2))
    u = mean[0] - b / (2 * np.pi) * dy * e
    v = mean[1] + b / (2 * np.pi) * dx * e
    T = 1.0 - (gamma - 1.0) * b * b / (8.0 * gamma * np.pi ** 2) * e * e
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    return rho, u, v, p


def vortex(n=512, seed=0, noise=0.01):
    """Isentropic vortex (strength 5, centre (5, 5), mean flow (1, 1)) on periodic [0, 10]^2
    with the density multiplied by (1 + noise * zeta), zeta ~ U[-1, 1]; u, v, p kept."""
    rho, u, v, p = vortex_primitive(n)
    g = SplitMix64(int(seed) * 15485863 + 11)
    zeta = g.uniform_array(n * n, -1.0, 1.0).reshape(n, n)
    rho0 = rho * (1.0 + noise * zeta)
    u0 = prim_to_cons(rho0, u, v, p, 1.4, 2)
    return Problem(f"vortex_{seed}", 2, 4, n, n, (0.0, 0.0), (10.0, 10.0), (0, 0), u0, 1,
                   extra={"u": u, "v": v, "p": p, "rho0": rho0})


def random_smooth_euler_2d(nx, ny, seed=0, periodic=True):
    """Smooth, positive 2D Euler data built from a few random Fourier modes (test input)."""
    g = SplitMix64(int(seed) * 31337 + 5)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    def field_(base, amp):
        f = np.full_like(X, base)
        for _ in range(3):
            kx, ky = g.integers(1, 3), g.integers(1, 3)
            ph = g.uniform(0, 2 * np.pi)
            f = f + amp * g.uniform(0.3, 1.0) * np.sin(2 * np.pi * (kx * X + ky * Y) + ph)
        return f
    rho = field_(1.0, 0.15)
    u = field_(0.3, 0.2)
    v = field_(-0.2, 0.2)
    p = field_(1.0, 0.15)
    u0 = prim_to_cons(rho, u, v, p, 1.4, 2)
    bc = (0, 0) if periodic else (1, 1)
    return Problem(f"smooth2d_{seed}", 2, 4, nx, ny, (0.0, 0.0), (1.0, 1.0), bc, u0, 1)


def rough_euler_2d(nx, ny, seed=0, amp=0.1):
    """2D Euler data with no smooth or constant stretch anywhere: the smooth field of
    random_smooth_euler_2d with an independent uniform perturbation of relative size amp
    in every cell's density and pressure (seeded), periodic.  Throughput context for the
    weight-dependent paths of the kernels (test and benchmark input)."""
    P = random_smooth_euler_2d(nx, ny, seed=seed, periodic=True)
    noise = np.random.default_rng(int(seed) * 7877 + 11).uniform(-amp, amp, size=(2, ny, nx))
    rho0 = P.u0[0]
    u = P.u0[1] / rho0
    v = P.u0[2] / rho0
    p = 0.4 * (P.u0[3] - 0.5 * rho0 * (u * u + v * v))
    rho = rho0 * (1.0 + noise[0])
    p = p * (1.0 + noise[1])
    u0 = prim_to_cons(rho, u, v, p, 1.4, 2)
    return Problem(f"rough2d_{seed}", 2, 4, nx, ny, (0.0, 0.0), (1.0, 1.0), (0, 0), u0, 1)


def random_smooth_euler_1d(n, seed=0, periodic=True):
    """Smooth, positive 1D Euler data from a few random Fourier modes (test input)."""
    g = SplitMix64(int(seed) * 6007 + 9)
    x = (np.arange(n) + 0.5) / n
    def field_(base, amp):
        f = np.full_like(x, base)
        for _ in range(3):
            k = g.integers(1, 3)
            f = f + amp * g.uniform(0.3, 1.0) * np.sin(2 * np.pi * k * x + g.uniform(0, 2 * np.pi))
        return f
    u0 = prim_to_cons(field_(1.0, 0.15), field_(0.3, 0.2), None, field_(1.0, 0.15), 1.4, 1)[:, None, :].copy()
    bc = (0, 0) if periodic else (1, 1)
    return Problem(f"smooth1d_{seed}", 1, 3, n, 1, (0.0, 0.0), (1.0, 1.0), bc, u0, 1)


def random_piecewise_euler_1d(n, seed=0, pieces=4, periodic=False):
    """Piecewise-constant 1D Euler data with seeded states (test input)."""
    g = SplitMix64(int(seed) * 7877 + 1)
    x = cell_centres(0.0, 1.0, n)
    cuts = np.sort([g.uniform() for _ in range(pieces - 1)])
    st = np.array([(g.uniform(0.1, 1.5), g.uniform(-1, 1), g.uniform(0.03, 1.5)) for _ in range(pieces)])
    seg = np.searchsorted(cuts, x, side="right")
    u0 = prim_to_cons(st[seg, 0], st[seg, 1], None, st[seg, 2], 1.4, 1)[:, None, :].copy()
    bc = (0, 0) if periodic else (1, 1)
    return Problem(f"piecewise1d_{seed}", 1, 3, n, 1, (0.0, 0.0), (1.0, 1.0), bc, u0, 1)
