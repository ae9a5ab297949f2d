"""The library's interface numerics, compiled for the host, against the oracle (no GPU).

`tests/host_numerics.cu` builds the double-precision device numerics of
`csrc/wcns_device.cuh` (projection, Eq. 5-15 interpolation and weights, the Eq. 20 map
with its ideal-plateau shortcuts, the Riemann solvers, the App. B split flux) as a host
library.  Host and device builds share the source; on the host the divisions are IEEE
divisions and the bit-pattern compares plain ones, so the device results differ only by
rounding (the GPU parity tests compare those).  Checked here, interface by interface:

* the midpoint flux of six stencil states agrees with the oracle's to 1e-13 over the
  option matrix (weights, fluxes, projection, both families, p = 1 and 2, 1D and 2D
  Euler) on smooth, shocked and random stencils, and the fallback flag agrees;
* the compiled default configuration (FIX = 1) gives the run-time-option path's flux
  bit for bit;
* on smooth stencils, where the plateau shortcuts return the ideal weights without
  evaluating Eq. 20, the final weights equal the oracle's full evaluation exactly, and
  stencils whose weights leave the plateau gradually get the full map's weights;
* the flux difference of Eq. 3 differentiates polynomial fluxes of degree up to 6
  exactly at the cell centre (closed form; the two-point difference of App. B, degree 2);
* the adjoint's reverse sweep of one interface flux (`interface_flux_vjp`,
  wcns_adjoint.cuh) is the transpose of the forward flux's derivative: dot products
  against fourth-order central differences of the host-built forward flux;
* the ghost cells of the boundary faces (`face_cell`, Sec. 4.3) follow their
  definitions: mirror cells with the normal momentum reversed at walls, the edge cell for
  outflow, the grid's wrap, fixed states, and the exact moving shock at ghost-cell centres.
"""
import ctypes
import os
import shutil
import subprocess
import tempfile
import zlib

import numpy as np
import pytest

import oracle
from paper_2306_09760_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = {"JS": 0, "Z": 1, "FE": 2, "PFE": 3, "M": 4}
FLUXES = {"LLF": 0, "ROE": 1, "HLLC": 2, "LLF_FROZEN": 3}
DP = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def host():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tempfile.mkdtemp()
    so = os.path.join(d, "libhostnum.so")
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-x", "cu", "-shared", "-Xcompiler",
                        "-fPIC", "-o", so, os.path.join(HERE, "host_numerics.cu")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = ctypes.CDLL(so)
    L.host_interface_flux.restype = ctypes.c_int
    L.host_interface_flux.argtypes = [ctypes.c_int] * 6 + [ctypes.c_double] * 3 + [ctypes.c_int, DP, DP]
    L.host_weno_side.restype = ctypes.c_double
    L.host_weno_side.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, DP, DP, DP]
    L.host_flux_difference.restype = ctypes.c_double
    L.host_flux_difference.argtypes = [ctypes.c_int, DP, ctypes.c_double]
    L.host_interface_flux_vjp.restype = ctypes.c_int
    L.host_face_cell.restype = ctypes.c_double
    L.host_face_cell.argtypes = ([DP, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                  ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), DP, DP]
                                 + [ctypes.c_double] * 9)
    L.host_interface_flux_vjp.argtypes = [ctypes.c_int] * 5 + [ctypes.c_double] * 3 + [DP, DP, DP]
    yield L
    shutil.rmtree(d, ignore_errors=True)


def _stencil(rng, nvar, kind):
    x = np.arange(6, dtype=np.float64)
    if kind == "smooth":
        ph = rng.uniform(0, 6)
        rho = 1 + 0.1 * np.sin(0.3 * x + ph)
        u = 0.3 + 0.1 * np.cos(0.2 * x + ph)
        v = -0.2 + 0.05 * np.sin(0.1 * x)
        p = 1 + 0.1 * np.sin(0.25 * x + 1 + ph)
    elif kind == "shock":
        j = rng.integers(1, 6)
        rho = np.where(x < j, 1.0, 0.125) * (1 + 0.01 * rng.normal(size=6))
        u = np.where(x < j, 0.75, -0.1)
        v = np.where(x < j, 0.1, -0.3)
        p = np.where(x < j, 1.0, 0.1)
    else:
        rho, u, v, p = (rng.uniform(0.5, 1.5, 6), rng.uniform(-0.5, 0.5, 6), rng.uniform(-0.5, 0.5, 6),
                        rng.uniform(0.3, 1.5, 6))
    U = inputs.prim_to_cons(rho, u, v, p, 1.4, 1 if nvar == 3 else 2)
    return np.ascontiguousarray(U.T)


def _lib_flux(host, S, nvar, weights, flux, ch, zp, family, fixed=0, xi=1e6, alpha=1.5):
    F = np.zeros(nvar)
    fb = host.host_interface_flux(nvar, WEIGHTS[weights], FLUXES[flux], int(ch), zp, family, xi, 1e-40, alpha,
                                  fixed, S.ctypes.data_as(DP), F.ctypes.data_as(DP))
    assert fb >= 0
    return F, bool(fb)


CASES = [(w, f, ch, 1, 0) for w in WEIGHTS for f in FLUXES for ch in (0, 1)]
CASES += [("FE", "HLLC", 1, 2, 0), ("Z", "ROE", 1, 2, 0), ("FE", "LLF", 1, 1, 1), ("FE", "LLF", 0, 2, 1),
          ("JS", "LLF", 1, 1, 1)]


@pytest.mark.parametrize("weights,flux,ch,zp,family", CASES)
def test_interface_flux_matches_the_oracle(host, weights, flux, ch, zp, family):
    rng = np.random.default_rng(zlib.crc32(repr((weights, flux, ch, zp, family)).encode()))
    fam = "WENO" if family else "WCNS"
    for nvar in (3, 4):
        for kind in ("smooth", "shock", "random"):
            for _ in range(4):
                S = _stencil(rng, nvar, kind)
                F, fb = _lib_flux(host, S, nvar, weights, flux, ch, zp, family)
                Fo, fbo = oracle.interface_flux(S, nvar, weights=weights, flux=flux, characteristic=bool(ch), zp=zp,
                                                family=fam, alpha=(1.5, 1.5))
                assert fb == fbo, (nvar, kind)
                assert np.abs(F - Fo).max() <= 1e-13 * (1 + np.abs(Fo).max()), (nvar, kind, F, Fo)


def test_compiled_default_configuration_equals_run_time_options(host):
    """FIX = 1 (FE, Z p = 1, renormalised, HLLC, characteristic, WCNS family) compiles the
    default configuration without its option branches; it must not change a bit."""
    rng = np.random.default_rng(7)
    for nvar in (3, 4):
        for kind in ("smooth", "shock", "random"):
            for _ in range(20):
                S = _stencil(rng, nvar, kind)
                a, fa = _lib_flux(host, S, nvar, "FE", "HLLC", 1, 1, 0, fixed=0)
                b, fb = _lib_flux(host, S, nvar, "FE", "HLLC", 1, 1, 0, fixed=1)
                assert fa == fb and np.array_equal(a, b), (nvar, kind)


@pytest.mark.parametrize("zp", [1, 2])
def test_plateau_shortcut_gives_the_full_maps_weights(host, zp):
    """Smooth stencils sit on the FE ideal plateaus, where the library returns the ideal
    weights without evaluating Eq. 20 (before the map and, for p = 1, before the Z ratios
    are formed); the oracle evaluates the map in full.  The final weights agree exactly;
    off the plateaus (a jump in the stencil) they agree to rounding."""
    rng = np.random.default_rng(11 + zp)
    x = np.arange(-2, 3, dtype=np.float64)
    on = 0
    for trial in range(400):
        a = rng.uniform(-1, 1, 4) * np.array([1.0, 1.0, 0.2, 0.02])
        v = a[0] + a[1] * x + a[2] * x ** 2 + a[3] * x ** 3
        if trial % 4 == 3:
            v[rng.integers(0, 5)] += rng.uniform(0.5, 2.0)
        wz, wf = np.zeros(3), np.zeros(3)
        val = host.host_weno_side(WEIGHTS["FE"], zp, 1e6, 1e-40, v.ctypes.data_as(DP), wz.ctypes.data_as(DP),
                                  wf.ctypes.data_as(DP))
        vo, wzo, wfo, _ = oracle.interp(v, weights="FE", zp=zp)
        if np.array_equal(wfo, [1 / 16, 10 / 16, 5 / 16]):
            on += 1
            np.testing.assert_array_equal(wf, wfo)
        else:
            np.testing.assert_allclose(wf, wfo, rtol=0, atol=1e-13)
        np.testing.assert_allclose(wz, wzo, rtol=0, atol=1e-13)
        assert abs(val - vo) <= 1e-13 * (1 + np.abs(v).max())
    assert on > 200  # most smooth stencils take the shortcut


@pytest.mark.parametrize("zp", [1, 2])
def test_weights_leaving_the_plateau_gradually(host, zp):
    """A bump of growing size on a linear stencil moves the Z weights continuously away from
    the ideal weights, through the edge of the plateau shortcuts' bounds and across the
    null points of Eq. 20: wherever the oracle's full map leaves the ideal weights, so does
    the library, and elsewhere the two agree."""
    x = np.arange(-2, 3, dtype=np.float64)
    left = 0
    for pos in range(5):
        for amp in np.geomspace(1e-5, 3.0, 300):
            v = 0.5 + 0.3 * x
            v[pos] += amp
            wz, wf = np.zeros(3), np.zeros(3)
            host.host_weno_side(WEIGHTS["FE"], zp, 1e6, 1e-40, v.ctypes.data_as(DP), wz.ctypes.data_as(DP),
                                wf.ctypes.data_as(DP))
            _, wzo, wfo, _ = oracle.interp(v, weights="FE", zp=zp)
            np.testing.assert_allclose(wz, wzo, rtol=0, atol=1e-13)
            # near a null point the map is steep (slope up to ~xi), so rounding of w moves it
            np.testing.assert_allclose(wf, wfo, rtol=0, atol=1e-8, err_msg=f"pos {pos} amp {amp}")
            left += not np.array_equal(wfo, [1 / 16, 10 / 16, 5 / 16])
    assert 100 < left < 1400  # both sides of the plateau edge are sampled


@pytest.mark.parametrize("family,degree", [(0, 6), (1, 2)])
def test_flux_difference_is_exact_on_polynomials(host, family, degree):
    """Eq. 3: with F the exact midpoint values of a polynomial flux of degree <= 6 (on a grid
    of h = 1/8 around x_i = 0.3), the difference equals -F'(x_i) up to rounding, and not
    for degree 7.  The two-point difference of App. B, -(F(x_i + h/2) - F(x_i - h/2)) / h,
    is exact up to degree 2."""
    rng = np.random.default_rng(3 + family)
    h, xi = 1.0 / 8, 0.3
    for _ in range(20):
        c = rng.uniform(-1, 1, degree + 1)
        Fx = lambda t: sum(ck * t ** k for k, ck in enumerate(c))
        dF = sum(k * ck * xi ** (k - 1) for k, ck in enumerate(c) if k > 0)
        f = np.array([Fx(xi + (m - 2.5) * h) for m in range(6)])
        got = host.host_flux_difference(family, f.ctypes.data_as(DP), 1.0 / h)
        assert abs(got + dF) <= 1e-12 * (1 + np.abs(c).sum()), (got, -dF)
    if family == 0:  # degree 7 is not exact: the scheme is sixth order
        c = np.zeros(8); c[7] = 1.0
        f = np.array([(xi + (m - 2.5) * h) ** 7 for m in range(6)])
        got = host.host_flux_difference(0, f.ctypes.data_as(DP), 1.0 / h)
        assert abs(got + 7 * xi ** 6) > 1e-8


@pytest.mark.parametrize("zp", [1, 2])
def test_random_cubics_around_the_plateau_bounds(host, zp):
    """Cubic stencils of random slope and curvature: their smoothness indicators differ by
    factors of order one, so many have every Z ratio near the plateau shortcuts' bound with
    weights on either side of the plateau's edge.  The library's final weights equal the
    oracle's full evaluation (exactly where that is the ideal weights).  Asked for the value
    alone, as the kernels ask, the library also tests the ratios before the weights are
    formed; the value still equals the oracle's."""
    rng = np.random.default_rng(20 + zp)
    x = np.arange(-2, 3, dtype=np.float64)
    ideal = [1 / 16, 10 / 16, 5 / 16]
    on = off = 0
    for _ in range(2000):
        a = rng.normal(size=4) * np.array([1.0, 1.0, rng.uniform(0, 0.5), rng.uniform(0, 0.2)])
        v = a[0] + a[1] * x + a[2] * x ** 2 + a[3] * x ** 3
        wz, wf = np.zeros(3), np.zeros(3)
        host.host_weno_side(WEIGHTS["FE"], zp, 1e6, 1e-40, v.ctypes.data_as(DP), wz.ctypes.data_as(DP),
                            wf.ctypes.data_as(DP))
        vo, _, wfo, _ = oracle.interp(v, weights="FE", zp=zp)
        if np.array_equal(wfo, ideal):
            on += 1
            np.testing.assert_array_equal(wf, wfo)
        else:
            off += 1
            np.testing.assert_allclose(wf, wfo, rtol=0, atol=1e-8)
        val = host.host_weno_side(WEIGHTS["FE"], zp, 1e6, 1e-40, v.ctypes.data_as(DP), None, None)
        assert abs(val - vo) <= 1e-8 * (1 + np.abs(v).max()), (v, val, vo)
    assert on > 200 and off > 200


@pytest.mark.parametrize("zp", [1, 2])
def test_ratio_bound_on_stencils_built_for_its_edge(host, zp):
    """The ratio bound of the plateau shortcut matters where the centre sub-stencil is far
    rougher than the outer two and those two differ a little: then every Z ratio is small
    while a weight leaves its plateau.  Stencils with first differences (1.4, 1, -1, d3)
    (and their mirror images) make IS_0 minimal for d1 = 1 and IS_1 five times larger,
    and sweeping d3 takes IS_2 / IS_0 from 1 to about 1.25, through the edge of the weight
    plateaus.  Asked for the value alone (the kernels' path, with the ratio tests), the
    library gives the oracle's value on every one of them."""
    off = 0
    for d3 in np.linspace(-1.4, -0.9, 500):
        for mirror in (False, True):
            d = np.array([1.4, 1.0, -1.0, d3])
            if mirror:
                d = -d[::-1]
            v = np.concatenate([[0.0], np.cumsum(d)])
            vo, _, wfo, _ = oracle.interp(v, weights="FE", zp=zp)
            off += not np.allclose(wfo, [1 / 16, 10 / 16, 5 / 16], rtol=0, atol=1e-12)
            val = host.host_weno_side(WEIGHTS["FE"], zp, 1e6, 1e-40, v.ctypes.data_as(DP), None, None)
            assert abs(val - vo) <= 1e-10, (d3, mirror, val, vo)
    assert off > 100  # the sweep crosses the plateau edge


VJP_CASES = [  # weights, p, xi, stencil noise, difference step, tolerance
    ("JS", 1, 1e6, 0.05, 1e-5, 2e-6), ("JS", 2, 1e6, 0.05, 1e-5, 2e-6), ("Z", 2, 1e6, 0.05, 1e-5, 2e-6),
    # at xi = 100 the map is steep next to the ideal weights: differences need small steps
    ("FE", 2, 100.0, 0.05, 1e-7, 2e-6), ("PFE", 2, 100.0, 0.05, 1e-7, 2e-6),
    # at xi = 1e6 the map is a staircase: smooth stencils sit on its flat plateaus
    ("FE", 1, 1e6, 0.0, 1e-6, 1e-7), ("FE", 2, 1e6, 0.0, 1e-6, 1e-7),
]


@pytest.mark.parametrize("weights,zp,xi,noise,step,tol", VJP_CASES)
def test_interface_flux_vjp_is_the_transposed_derivative(host, weights, zp, xi, noise, step, tol):
    """<Sb, dS> with Sb = (dF/dS)^T Fb from the reverse sweep equals <Fb, dF/dS dS> from
    central differences of the forward flux (LLF with frozen alpha, the adjoint's flux;
    eps = 1e-6 as in the adjoint tests, where the Z weights stay differentiable).  A sample
    whose difference quotients at two steps disagree has a switch (the PFE box, a kink of
    the weights) within the step and is skipped; at most a quarter are."""
    rng = np.random.default_rng(zlib.crc32(repr((weights, zp, xi)).encode()))
    x = np.arange(6, dtype=np.float64)

    def flux(S, nvar, ch):
        F = np.zeros(nvar)
        S = np.ascontiguousarray(S)
        host.host_interface_flux(nvar, WEIGHTS[weights], FLUXES["LLF_FROZEN"], ch, zp, 0, xi, 1e-6, 1.7, 0,
                                 S.ctypes.data_as(DP), F.ctypes.data_as(DP))
        return F

    def quotient(S, dS, nvar, ch, e):
        return (-flux(S + 2 * e * dS, nvar, ch) + 8 * flux(S + e * dS, nvar, ch)
                - 8 * flux(S - e * dS, nvar, ch) + flux(S - 2 * e * dS, nvar, ch)) / (12 * e)

    checked = skipped = 0
    for nvar in (3, 4):
        for ch in (0, 1):
            for _ in range(8):
                ph = rng.uniform(0, 6)
                rho = 1 + 0.2 * np.sin(0.5 * x + ph) + noise * rng.normal(size=6)
                u = 0.3 + 0.2 * np.cos(0.4 * x + ph)
                v = 0.1 * np.sin(0.3 * x)
                p = 1 + 0.2 * np.sin(0.45 * x + 1)
                S = np.ascontiguousarray(inputs.prim_to_cons(rho, u, v, p, 1.4, 1 if nvar == 3 else 2).T)
                Fb, dS = rng.normal(size=nvar), rng.normal(size=S.shape)
                Sb = np.zeros_like(S)
                assert host.host_interface_flux_vjp(nvar, WEIGHTS[weights], FLUXES["LLF_FROZEN"], ch, zp, xi, 1e-6,
                                                    1.7, S.ctypes.data_as(DP), Fb.ctypes.data_as(DP),
                                                    Sb.ctypes.data_as(DP)) == 0
                scale = 1e-3 * np.abs(Fb).sum()
                rhs = (Fb * quotient(S, dS, nvar, ch, step)).sum()
                rhs2 = (Fb * quotient(S, dS, nvar, ch, step / 2)).sum()
                if abs(rhs - rhs2) > tol * (abs(rhs2) + scale):
                    skipped += 1
                    continue
                checked += 1
                lhs = (Sb * dS).sum()
                assert abs(lhs - rhs2) <= tol * (abs(rhs2) + scale), (nvar, ch, lhs, rhs2)
    assert skipped * 3 <= checked, (checked, skipped)


@pytest.mark.parametrize("weights", list(WEIGHTS))
@pytest.mark.parametrize("family", [0, 1])
def test_scalar_advection_flux_matches_the_oracle(host, weights, family):
    """u_t + a u_x = 0 (Sec. 2): the upwind interpolated state times a (WCNS family) or the
    split flux reconstruction (App. B), for a of both signs, on smooth, jump and random
    stencils."""
    rng = np.random.default_rng(zlib.crc32(repr((weights, family)).encode()))
    x = np.arange(6, dtype=np.float64)
    for a in (1.0, -0.7):
        for kind in range(3):
            for _ in range(10):
                if kind == 0:
                    S = np.sin(0.4 * x + rng.uniform(0, 6))
                elif kind == 1:
                    S = np.where(x < rng.integers(1, 6), 1.0, 0.0) + 0.01 * rng.normal(size=6)
                else:
                    S = rng.normal(size=6)
                S = np.ascontiguousarray(S.reshape(6, 1))
                F = np.zeros(1)
                host.host_interface_flux(1, WEIGHTS[weights], 0, 0, 1, family, 1e6, 1e-40, a, 0,
                                         S.ctypes.data_as(DP), F.ctypes.data_as(DP))
                Fo, _ = oracle.interface_flux(S, 1, system=0, ax=a, weights=weights,
                                              family="WENO" if family else "WCNS")
                assert abs(F[0] - Fo[0]) <= 1e-13 * (1 + abs(Fo[0])), (a, kind, F, Fo)


FACE_GRID, FACE_TRANS, FACE_WALL, FACE_FIXED, FACE_FIXED_THEN_WALL, FACE_SHOCK = range(6)


def test_boundary_face_ghost_cells_follow_their_definitions(host):
    nx, ny, pitch, nv = 13, 9, 16, 4
    rng = np.random.default_rng(8)
    u = np.ascontiguousarray(rng.uniform(0.5, 2.0, size=(nv, ny, pitch)))
    lo, hx, hy = (0.1, -0.2), 1.0 / nx, 0.5 / ny
    ua, ub = np.array([8.0, 57.1, -33.0, 563.5]), np.array([1.4, 0.0, 0.0, 2.5])
    wall_x, x0, dxdy, speed, time = 1.0 / 6.0 + 0.1, 0.3, 1.0 / np.sqrt(3.0), 20.0, 0.013
    tarr = (ctypes.c_int * 4)
    cases = [(FACE_TRANS, FACE_WALL, FACE_FIXED_THEN_WALL, FACE_SHOCK), (FACE_FIXED, FACE_GRID, FACE_WALL, FACE_TRANS),
             (FACE_GRID, FACE_GRID, FACE_GRID, FACE_GRID)]
    for types in cases:
        for dir_, n, nlines in ((0, nx, ny), (1, ny, nx)):
            for bc in (0, 1):
                if bc == 0 and any(t != FACE_GRID for t in types):
                    continue  # periodic lines have no faces
                for line in range(nlines):
                    for m in list(range(-3, 0)) + list(range(n, n + 3)) + [0, n - 1]:
                        for v in range(nv):
                            got = host.host_face_cell(u.ctypes.data_as(DP), pitch, ny * pitch, dir_, line, m, n, bc, v,
                                                      tarr(*types), ua.ctypes.data_as(DP), ub.ctypes.data_as(DP),
                                                      wall_x, x0, dxdy, speed, lo[0], lo[1], hx, hy, time)

                            def cell(k):
                                return u[v, line, k] if dir_ == 0 else u[v, k, line]

                            typ = types[2 * dir_ + (0 if m < 0 else 1)]
                            # ghost-cell centre
                            x = lo[0] + ((m if dir_ == 0 else line) + 0.5) * hx
                            y = lo[1] + ((line if dir_ == 0 else m) + 0.5) * hy
                            if 0 <= m < n:
                                want = cell(m)
                            elif typ == FACE_GRID:
                                want = cell(m % n) if bc == 0 else cell(min(max(m, 0), n - 1))
                            elif typ == FACE_TRANS:
                                want = cell(min(max(m, 0), n - 1))
                            elif typ == FACE_FIXED or (typ == FACE_FIXED_THEN_WALL and x < wall_x):
                                want = ua[v]
                            elif typ in (FACE_WALL, FACE_FIXED_THEN_WALL):
                                mirror = -1 - m if m < 0 else 2 * n - 1 - m
                                want = -cell(mirror) if v == 1 + dir_ else cell(mirror)
                            else:  # moving oblique shock: state a behind x0 + (y + speed t) dxdy
                                want = ua[v] if x < x0 + (y + speed * time) * dxdy else ub[v]
                            assert got == want, (types, dir_, bc, line, m, v, got, want)
