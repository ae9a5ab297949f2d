"""Degenerate and extreme grid sizes through the C ABI against the oracle: lines shorter
than the stencil, single cells, one-row 2D grids, many independent lines, and a line of
four million cells checked on sampled cells."""
import numpy as np
import pytest

import oracle
from paper_2306_09760_gb300 import inputs
from parity import check64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2306_09760_gb300 import build as wbuild
    wbuild.build()
    from paper_2306_09760_gb300 import wcns
    wcns.load()
    return wcns


def gpu_rhs(W, P, dtype, **params):
    import torch
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        S = W.Solver(P, dtype, stream=stream, **params)
        L = S.numpy(S.rhs()).astype(np.float64)
        st, _ = S.status()
        S.close()
    assert st == W.WCNS_OK
    return L


def euler1d(n, seed, bc):
    P = inputs.random_smooth_euler_1d(max(n, 8), seed=seed, periodic=(bc == 0))
    u0 = P.u0[:, :, :n].copy()
    return inputs.Problem("tiny", 1, 3, n, 1, (0.0, 0.0), (float(n), 1.0), (bc, bc), u0, 1)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 11])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("family", ["WCNS", "WENO"])
def test_lines_shorter_than_the_stencil(W, n, bc, family):
    P = euler1d(n, seed=n, bc=bc)
    L = gpu_rhs(W, P, "f64", family=family)
    Lr, _ = oracle.rhs(P, family=family)
    check64(L, Lr, lambda u0: oracle.rhs(P, u0, family=family)[0], P.u0, f"n={n} bc={bc}", strict=True)
    L32 = gpu_rhs(W, P, "f32", family=family)
    scale = max(np.abs(Lr).mean(), 1e-30)
    assert np.abs(L32 - Lr).mean() / scale < 1e-4 or np.abs(L32 - Lr).max() < 1e-5 * np.abs(P.u0).max()


@pytest.mark.parametrize("n", [1, 4, 6])
def test_advection_tiny(W, n):
    x = -1.0 + np.arange(n) * (2.0 / n)
    P = inputs.Problem("a", 1, 1, n, 1, (-1.0, 0.0), (1.0, 1.0), (0, 0),
                       np.sin(np.pi * x)[None, None, :].copy() + 0.3, 0, adv_speed=(1.0, 0.0))
    L = gpu_rhs(W, P, "f64")
    Lr, _ = oracle.rhs(P)
    check64(L, Lr, lambda u0: oracle.rhs(P, u0)[0], P.u0, f"adv n={n}", strict=True)


@pytest.mark.parametrize("nx,ny", [(1, 1), (3, 2), (1, 9), (9, 1), (260, 1), (1, 260)])
def test_thin_2d_grids(W, nx, ny):
    Q = inputs.random_smooth_euler_2d(max(nx, 8), max(ny, 8), seed=nx * 31 + ny)
    P = inputs.Problem("thin", 2, 4, nx, ny, (0.0, 0.0), (1.0, 1.0), (1, 0), Q.u0[:, :ny, :nx].copy(), 1)
    L = gpu_rhs(W, P, "f64")
    Lr, _ = oracle.rhs(P)
    check64(L, Lr, lambda u0: oracle.rhs(P, u0)[0], P.u0, f"{nx}x{ny}", strict=True)


# 1224 rows give at least two waves of four-interface x blocks (1019-cell tiles) on a
# 152-SM GPU, so those grids take that form; 9 rows keep one interface per thread
# (251-cell tiles).
@pytest.mark.parametrize("nx,ny", [(5, 1224), (6, 1224), (1018, 1224), (1019, 1224), (1020, 1224),
                                   (2038, 1224), (2039, 1224), (2040, 1224),
                                   (250, 9), (251, 9), (252, 9), (503, 9)])
@pytest.mark.parametrize("bc", [0, 1])
def test_f32_x_tile_boundaries(W, nx, ny, bc):
    """Single-precision 2D RHS at and around the x tiles of the single-precision sweep,
    periodic and transmissive."""
    Q = inputs.random_smooth_euler_2d(nx, ny, seed=nx + 7 * bc, periodic=(bc == 0))
    L = gpu_rhs(W, Q, "f32")
    Lr, _ = oracle.rhs(Q)
    err = np.abs(L - Lr)
    assert np.all(np.isfinite(L))
    assert err.mean() / np.abs(Lr).mean() < 3e-4, err.mean() / np.abs(Lr).mean()
    # a misplaced cell or ghost would show as an O(|L|) error at the tile edges
    assert err.max() < 3e-3 * np.abs(Lr).max(), (err.max(), np.unravel_index(err.argmax(), err.shape))


def test_many_independent_lines(W):
    """ndim = 1 with ny > 1: every row is its own line (no coupling between rows)."""
    nx, ny = 300, 517
    rng = np.random.default_rng(4)
    lines = [inputs.random_piecewise_euler_1d(nx, seed=int(s)).u0[:, 0, :] for s in rng.integers(0, 10 ** 6, ny)]
    u0 = np.stack(lines, axis=1)
    P = inputs.Problem("lines", 1, 3, nx, ny, (0.0, 0.0), (1.0, 1.0), (1, 1), u0, 1)
    L = gpu_rhs(W, P, "f64")
    for j in (0, 1, 250, ny - 1):
        Q = inputs.Problem("line", 1, 3, nx, 1, (0.0, 0.0), (1.0, 1.0), (1, 1), u0[:, j:j + 1, :].copy(), 1)
        Lr, _ = oracle.rhs(Q)
        check64(L[:, j:j + 1, :], Lr, lambda v: oracle.rhs(Q, v)[0], Q.u0, f"line {j}", strict=True)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_four_million_cell_line(W, dtype):
    """A 1D line of 2^22 + 123 cells (ragged last tile), transmissive, with data that varies
    on the scale of a few hundred cells (unit cells, so single precision still resolves
    the flux differences): sampled cells against the oracle's per-cell RHS."""
    n = (1 << 22) + 123
    i = np.arange(n, dtype=np.float64)
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * i / 517.0) + 0.1 * np.sin(2 * np.pi * i / 91.0)
    vel = 0.3 * np.sin(2 * np.pi * i / 313.0)
    p = 1.0 + 0.2 * np.cos(2 * np.pi * i / 211.0)
    u0 = inputs.prim_to_cons(rho[None, :], vel[None, :], None, p[None, :], 1.4, 1)
    P = inputs.Problem("long", 1, 3, n, 1, (0.0, 0.0), (float(n), 1.0), (1, 1), u0, 1)
    L = gpu_rhs(W, P, dtype)
    rng = np.random.default_rng(3)
    cells = np.concatenate([rng.integers(0, n, 400), [0, 1, 2, n - 3, n - 2, n - 1]])
    ref = oracle.rhs_cells(P, P.u0, cells)
    got = L[:, 0, cells].T
    if dtype == "f64":
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < 1e-11, err  # one evaluation: no round-off allowance
    else:
        err = np.abs(got - ref)
        assert err.mean() / np.abs(ref).mean() < 1e-4
        assert err.max() < 3e-3 * np.abs(ref).max(), (err.max(), cells[err.max(axis=1).argmax()])


def _line_sizes(kind):
    """Line lengths around the x sweep's choice of block width: lines whose 256-thread
    tiles (251 cells) would give fewer blocks than SMs run 32-thread blocks (27 cells)."""
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    return {"narrow_ragged": 27 * 37 + 13, "narrow_widest": (nsm - 1) * 251,
            "wide_narrowest": nsm * 251, "narrow_one_tile": 27, "narrow_two_tiles": 28}[kind]


@pytest.mark.parametrize("kind", ["narrow_ragged", "narrow_widest", "wide_narrowest",
                                  "narrow_one_tile", "narrow_two_tiles"])
@pytest.mark.parametrize("system", ["advection", "euler1d"])
@pytest.mark.parametrize("bc", [0, 1])
def test_x_block_width_choice(W, kind, system, bc):
    """One-dimensional RHS on both sides of the narrow/wide block choice, FP64 against the
    oracle (1e-11 or the oracle's own round-off sensitivity) and FP32 by the relative L1
    bound of the other single-precision line tests."""
    n = _line_sizes(kind)
    # periodic data varying over a few hundred cells at every length (unit cells), so
    # single precision still resolves the flux differences
    i = np.arange(n, dtype=np.float64)
    k1, k2, k3 = max(1, n // 300), max(1, n // 97), max(1, n // 211)
    wave = lambda k, ph: np.sin(2 * np.pi * k * i / n + ph)
    if system == "euler1d":
        rho = 1.0 + 0.2 * wave(k1, 0.3) + 0.05 * wave(k2, 1.1)
        vel = 0.3 * wave(k3, 2.0)
        p = 1.0 + 0.2 * wave(k2, 0.7)
        u0 = inputs.prim_to_cons(rho[None, :], vel[None, :], None, p[None, :], 1.4, 1)
        P = inputs.Problem("line", 1, 3, n, 1, (0.0, 0.0), (float(n), 1.0), (bc, bc), u0, 1)
    else:
        u0 = wave(k1, 0.0) + 0.25 * wave(k2, 0.5) + 0.3
        P = inputs.Problem("a", 1, 1, n, 1, (0.0, 0.0), (float(n), 1.0), (bc, bc), u0[None, None, :].copy(), 0,
                           adv_speed=(1.0, 0.0))
    Lr, _ = oracle.rhs(P)
    L = gpu_rhs(W, P, "f64")
    check64(L, Lr, lambda u0: oracle.rhs(P, u0)[0], P.u0, f"{system} n={n} bc={bc}", strict=True)
    L32 = gpu_rhs(W, P, "f32")
    assert np.all(np.isfinite(L32))
    err = np.abs(L32 - Lr)
    print(f"\n{system} n={n} bc={bc} FP32 RHS: max / max|L| {err.max() / np.abs(Lr).max():.2e}")
    assert err.mean() / np.abs(Lr).mean() < 1e-4, err.mean() / np.abs(Lr).mean()
    # measured at most 5.9e-5 (1D Euler, 37901 cells); a misplaced ghost or tile-edge cell
    # would put an error of the order of max|L| there
    assert err.max() < 1e-3 * np.abs(Lr).max(), (err.max() / np.abs(Lr).max(), err.argmax())


def test_fp64_device_reciprocal_against_ieee(W):
    """Every double-precision division of the sweeps goes through the library's reciprocal
    (two Newton steps from the reciprocal unit's approximation): over values spread across
    the normal range it is within 2 ulp of the IEEE reciprocal, and exact on powers of two."""
    import torch
    rng = np.random.default_rng(12)
    mant = rng.uniform(1.0, 2.0, 400000)
    expo = rng.integers(-1000, 1000, 400000)
    x = np.ldexp(mant, expo) * rng.choice([-1.0, 1.0], 400000)
    x = np.concatenate([x, np.ldexp(1.0, np.arange(-1020, 1021)), [1.0, 3.0, 10.0, 1.0 / 3.0, 0.1, 1e300, 1e-300]])
    xd = torch.as_tensor(x, device="cuda")
    out = torch.empty_like(xd)
    W.wcns_reciprocal_f64(xd, out)
    torch.cuda.synchronize()
    r = out.cpu().numpy()
    ref = 1.0 / x
    ulps = np.abs(r - ref) / np.spacing(np.abs(ref))
    print(f"\nFP64 device reciprocal: max error {ulps.max():.2f} ulp, mean {ulps.mean():.3f}")
    assert ulps.max() <= 2.0, ulps.max()
    pw = np.ldexp(1.0, np.arange(-1020, 1021))
    np.testing.assert_array_equal(r[400000:400000 + len(pw)], 1.0 / pw)
