"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it checks.  None of them re-types the oracle's own
formula: they compare it with printed values (Table 1, Eq. 18), closed forms (the
linear scheme's Fourier symbol, RK amplification polynomials, polynomial exactness,
the exact Riemann solution), invariants (conservation, symmetry) and finite
differences.
"""
from fractions import Fraction
import math
import os

import numpy as np
import pytest

import oracle
from oracle import exact_riemann
from paper_2306_09760_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _frac(s):
    return float(Fraction(s))


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------------------
# FE mapping function: Eq. 20-21 with Table 2, pinned by Table 1
# ---------------------------------------------------------------------------
def test_table1_control_values_at_large_xi():
    """Table 1: the map sends every control point to its control value (xi = 1e6, kappa = 0.5)."""
    for case, i, orig, mapped in _golden("table1_control_values.txt"):
        g = oracle.fe_map(int(i), _frac(orig), xi=1e6, kappa=0.5)
        assert abs(g - _frac(mapped)) <= 1e-15, (case, i, orig, g)
    for i in range(3):  # weights that vanish stay zero (the "-" entries of Table 1)
        assert oracle.fe_map(i, 0.0) == 0.0


# Null points kappa*(psi_j + psi_{j-1}) at kappa = 1/2: midpoints of consecutive control
# points of Table 2 (0, then the Table 1 control points, then 1).
NULLS = {0: [1 / 32, (1 / 16 + 1 / 11) / 2, (1 / 11 + 1) / 2],
         1: [10 / 32, (10 / 16 + 2 / 3) / 2, (2 / 3 + 10 / 11) / 2, (10 / 11 + 1) / 2],
         2: [5 / 32, (5 / 16 + 1 / 3) / 2, (1 / 3 + 1) / 2]}


def test_fe_map_is_a_staircase():
    """Eq. 20 at xi = 1e6: flat at the control values between consecutive null points
    kappa*(psi_j + psi_{j-1}) and the identity below the first and above the last."""
    nulls = NULLS
    plateaus = {0: [1 / 16, 1 / 6], 1: [10 / 16, 1 / 2, 5 / 6], 2: [5 / 16, 1 / 2]}
    rng = np.random.default_rng(1)
    for i in range(3):
        z = nulls[i]
        for w in rng.uniform(0, 1, 400):
            if min(abs(w - zz) for zz in z) < 1e-4:
                continue
            k = sum(w > zz for zz in z)
            expect = w if k in (0, len(z)) else plateaus[i][k - 1]
            assert abs(oracle.fe_map(i, w) - expect) < 1e-14
            # flat means zero slope, identity means unit slope
            assert abs(oracle.fe_map_deriv(i, w) - (1.0 if k in (0, len(z)) else 0.0)) < 1e-12


def test_fe_map_endpoints_and_monotone():
    """g(0) = 0 and g(1) = 1 once the tanh terms saturate (xi = 1e6), approximately at the
    paper's xi = 100."""
    for i in range(3):
        for xi, tol in ((100.0, 1e-3), (1e6, 1e-15)):
            assert abs(oracle.fe_map(i, 0.0, xi=xi)) < tol
            assert abs(oracle.fe_map(i, 1.0, xi=xi) - 1.0) < tol
        # away from the null points the xi = 100 map is within 1e-3 of the xi = 1e6 staircase
        for w in np.linspace(0, 1, 2001):
            if min(abs(w - z) for z in NULLS[i]) > 0.05:
                assert abs(oracle.fe_map(i, w, xi=100.0) - oracle.fe_map(i, w, xi=1e6)) < 1e-3


def test_fe_map_kappa_below_half_misses_control_values():
    """Sec. 3.2 (Fig. 5 discussion): with kappa = 0.3 the map no longer reaches the control
    value at the control point, which is why kappa = 0.5 is chosen."""
    assert abs(oracle.fe_map(1, 2 / 3, kappa=0.3) - 0.5) > 1e-2
    assert abs(oracle.fe_map(1, 2 / 3, kappa=0.5) - 0.5) < 1e-15


def test_m_map_properties():
    """Eq. 13 (Henrick): g(0) = 0, g(d) = d, g(1) = 1 and g'(d) = 0."""
    for d in (1 / 16, 10 / 16, 5 / 16):
        assert abs(oracle.m_map(0.0, d)) < 1e-16
        assert abs(oracle.m_map(d, d) - d) < 1e-15
        assert abs(oracle.m_map(1.0, d) - 1.0) < 1e-14
        e = 1e-6
        slope = (oracle.m_map(d + e, d) - oracle.m_map(d - e, d)) / (2 * e)
        assert abs(slope) < 1e-5


# ---------------------------------------------------------------------------
# Interpolation: Eq. 5-6 with the weights, pinned by polynomial exactness and Eq. 18
# ---------------------------------------------------------------------------
X5 = np.arange(-2, 3, dtype=np.float64)  # stencil nodes x_{i-2}..x_{i+2} (h = 1, x_i = 0)


def _interp(f, **kw):
    return oracle.interp(f(X5), **kw)


def test_ideal_weights_recovered_and_degree4_exact():
    """Sec. 3.1 Case0: on smooth data the FE map returns the ideal weights (1/16, 10/16, 5/16)
    exactly, and the interpolant reproduces polynomials of degree 4 at x_{i+1/2}."""
    rng = np.random.default_rng(2)
    for _ in range(50):
        a = rng.uniform(-1, 1, 5) * np.array([1.0, 100.0, 0.5, 0.05, 0.005])
        f = lambda x: a[0] + a[1] * x + a[2] * x ** 2 + a[3] * x ** 3 + a[4] * x ** 4
        val, wz, wf, mapped = _interp(f, weights="FE")
        assert mapped == 1
        np.testing.assert_allclose(wf, [1 / 16, 10 / 16, 5 / 16], rtol=0, atol=2e-16)
        assert abs(val - f(0.5)) < 1e-12 * (1 + abs(a).sum())
        assert np.all(np.abs(wz - [1 / 16, 10 / 16, 5 / 16]) < 0.01)


def _case_data(case, A=1.0, B=0.0, n=4, J=1e6):
    """Linear-plus-monomial data f = A x + B x^n / n! with a jump of size J placed in the
    interval that defines each case of Sec. 3.1."""
    f = lambda x: A * x + B * x ** n / math.factorial(n)
    v = f(X5).copy()
    jump = {"Case1": [0], "Case2": [0, 1], "Case3": [3, 4], "Case4": [4]}.get(case, [])
    v[jump] += J
    return v, f


@pytest.mark.parametrize("case,n", [(r[0], int(r[1])) for r in _golden("eq18_truncation.txt")])
def test_eq18_truncation_coefficients(case, n):
    """Eq. 18: the embedded combinations selected by the FE weights have the printed leading
    truncation errors (exact minus interpolated value = coefficient * h^n f^(n))."""
    coef = {r[0]: _frac(r[2]) for r in _golden("eq18_truncation.txt")}[case]
    B = 1e-2 if case != "Case0" else 1.0
    A = 1.0 if case != "Case0" else 1e3
    v, f = _case_data(case, A=A, B=B, n=n)
    val, wz, wf, mapped = oracle.interp(v, weights="FE", zp=2)
    err = f(0.5) - val
    assert abs(err - coef * B) < 1e-6 * abs(coef * B), (case, err, coef * B, wf)


def test_embedded_weights_case1_case4():
    """Table 1 Case1/Case4: the Z weights sit at the control points and the FE weights at the
    control values (1/2, 1/2) and (1/6, 5/6)."""
    v, _ = _case_data("Case1", B=1e-2)
    _, wz, wf, _ = oracle.interp(v, weights="FE", zp=2)
    assert abs(wz[1] - 2 / 3) < 5e-3 and abs(wz[2] - 1 / 3) < 5e-3
    np.testing.assert_allclose(wf, [0, 0.5, 0.5], atol=1e-14)
    v, _ = _case_data("Case4", B=1e-2)
    _, wz, wf, _ = oracle.interp(v, weights="FE", zp=2)
    assert abs(wz[0] - 1 / 11) < 5e-3 and abs(wz[1] - 10 / 11) < 5e-3
    np.testing.assert_allclose(wf, [1 / 6, 5 / 6, 0], atol=1e-14)


def test_weight_families_and_pfe_switch():
    """Eq. 11 (JS), Eq. 14 (Z), Eq. 12-13 (M) are convex weights; App. A: the PFE switch keeps
    the Z weights inside the box |w_k - d_k| <= cv and maps them outside."""
    rng = np.random.default_rng(3)
    for _ in range(100):
        v = rng.normal(size=5)
        for kind in ("JS", "Z", "M", "FE", "PFE"):
            _, _, wf, _ = oracle.interp(v, weights=kind)
            assert abs(wf.sum() - 1.0) < 1e-14 and np.all(wf >= -1e-15)
    f = lambda x: 1 + 10 * x + 0.3 * x ** 2 + 0.01 * x ** 3
    _, wz, wf, mapped = oracle.interp(f(X5), weights="PFE", cv=1.0)
    assert mapped == 0 and np.array_equal(wz, wf)
    _, wz, wf, mapped = oracle.interp(f(X5), weights="PFE", cv=0.0)
    assert mapped == 1
    np.testing.assert_allclose(wf, [1 / 16, 10 / 16, 5 / 16], rtol=0, atol=2e-16)


# ---------------------------------------------------------------------------
# Whole RHS for scalar advection: Eq. 2-3 with Eq. 5-6, pinned by the Fourier symbol
# ---------------------------------------------------------------------------
D3 = (75 / 64, -25 / 384, 3 / 640)
C5 = np.array([3, -20, 90, 60, -5]) / 128.0


def _adv_problem(n, u0, L=None, c=1.0):
    L = float(n) if L is None else L
    return inputs.Problem("adv", 1, 1, n, 1, (0.0, 0.0), (L, 1.0), (0, 0),
                          np.asarray(u0, dtype=np.float64)[None, None, :].copy(), 0, adv_speed=(c, 0.0))


def symbol(alpha, h=1.0, c=1.0):
    """Eigenvalue of the linear (ideal-weight) scheme for the mode e^{i alpha j}:
    lambda = -(c/h) C(alpha) sum_m d_m (e^{i alpha (m-1)} - e^{-i alpha m}),
    C(alpha) = sum_{l=-2..2} c_l e^{i alpha l} with c = (3, -20, 90, 60, -5)/128."""
    C = sum(C5[l + 2] * np.exp(1j * alpha * l) for l in range(-2, 3))
    S = sum(D3[m - 1] * (np.exp(1j * alpha * (m - 1)) - np.exp(-1j * alpha * m)) for m in (1, 2, 3))
    return -(c / h) * C * S


def test_eq3_consistency():
    """Eq. 3 is a consistent first derivative: d1 + 3 d2 + 5 d3 = 1 (exact fractions)."""
    d = [Fraction(75, 64), Fraction(-25, 384), Fraction(3, 640)]
    assert d[0] + 3 * d[1] + 5 * d[2] == 1


@pytest.mark.parametrize("k", [1, 2, 3])
def test_linear_fourier_symbol(k):
    """Sec. 3.2 (Eq. 22-28) linear special case: with the weights on the ideal plateau
    (xi = 1e6) the RHS of a resolved sine equals the closed-form modified wavenumber."""
    n = 64
    alpha = 2 * np.pi * k / n
    j = np.arange(n)
    for part in ("sin", "cos"):
        u0 = np.sin(alpha * j) if part == "sin" else np.cos(alpha * j)
        P = _adv_problem(n, u0 + 2.0)  # offset keeps the data away from zero; constants are exact
        L, nonph = oracle.rhs(P)
        lam = symbol(alpha)
        ex = lam * np.exp(1j * alpha * j)
        expect = ex.imag if part == "sin" else ex.real
        assert np.max(np.abs(L[0, 0] - expect)) < 2e-13


def test_rk3_and_rk4_amplification():
    """TVD-RK3 and Eq. 16 (classical RK4) amplify a linear mode by the Taylor polynomials of
    exp(z) of degree 3 and 4, z = dt * lambda."""
    n, k = 64, 2
    alpha = 2 * np.pi * k / n
    j = np.arange(n)
    lam = symbol(alpha)
    dt = 0.5
    z = dt * lam
    for rk4, deg in ((False, 3), (True, 4)):
        P = _adv_problem(n, np.sin(alpha * j) + 2.0)
        u, t, taken, _ = oracle.step(P, dt=dt, nsteps=1, rk4=rk4)
        amp = sum(z ** m / math.factorial(m) for m in range(deg + 1))
        expect = (amp * np.exp(1j * alpha * j)).imag + 2.0
        assert np.max(np.abs(u[0, 0] - expect)) < 1e-13


def test_spatial_order_five_at_large_xi():
    """Fifth-order convergence of the RHS for smooth advection at xi = 1e6 (Sec. 3.1, Case0),
    and the lower order of the xi = 100 map, whose plateau misses the ideal weights."""
    errs = {}
    for xi in (1e6, 100.0):
        e = []
        for n in (40, 80, 160, 320):
            x = -1.0 + np.arange(n) * (2.0 / n)
            P = _adv_problem(n, np.sin(np.pi * x), L=2.0)
            L, _ = oracle.rhs(P, xi=xi)
            e.append(np.max(np.abs(L[0, 0] + np.pi * np.cos(np.pi * x))))
        errs[xi] = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert np.all(errs[1e6] > 4.8) and np.all(errs[1e6] < 5.3), errs
    assert np.all(errs[100.0] < 3.6), errs


def test_periodic_conservation_advection():
    """Eq. 3 telescopes: on a periodic grid sum_i L_i = 0 to round-off (also for shocks)."""
    rng = np.random.default_rng(5)
    u0 = np.where(rng.uniform(size=100) > 0.5, 1.0, 0.0) + 0.1 * rng.normal(size=100)
    P = _adv_problem(100, u0)
    L, _ = oracle.rhs(P)
    assert abs(L.sum()) < 1e-13 * np.abs(L).sum()


# ---------------------------------------------------------------------------
# Euler: eigenvectors, Riemann fluxes, conservation, exact solution, symmetry
# ---------------------------------------------------------------------------
def _flux_x(U, g=1.4):
    nv = len(U)
    rho, mx = U[0], U[1]
    u = mx / rho
    if nv == 4:
        v = U[2] / rho
        E = U[3]
        p = (g - 1) * (E - 0.5 * rho * (u * u + v * v))
        return np.array([mx, mx * u + p, U[2] * u, (E + p) * u])
    E = U[2]
    p = (g - 1) * (E - 0.5 * rho * u * u)
    return np.array([mx, mx * u + p, (E + p) * u])


@pytest.mark.parametrize("nvar", [3, 4])
def test_eigenvectors_diagonalise_fd_jacobian(nvar):
    """The characteristic projection uses left/right eigenvectors of dF/dU: L R = I and
    L A R = diag(u - c, u, [u,] u + c), with A from central differences of F."""
    rng = np.random.default_rng(7)
    g = 1.4
    for _ in range(10):
        rho, u, v, p = rng.uniform(0.2, 2), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.1, 2)
        if nvar == 3:
            v = 0.0
        U = inputs.prim_to_cons(rho, u, v, p, g, 1 if nvar == 3 else 2)
        c = math.sqrt(g * p / rho)
        H = (U[-1] + p) / rho
        R, L = oracle.eigenvectors(nvar, g, u, v, H, c)
        np.testing.assert_allclose(L @ R, np.eye(nvar), atol=1e-13)
        A = np.zeros((nvar, nvar))
        for k in range(nvar):
            e = np.zeros(nvar); e[k] = 1e-6 * max(1.0, abs(U[k]))
            A[:, k] = (_flux_x(U + e) - _flux_x(U - e)) / (2 * e[k])
        lam = [u - c, u, u + c] if nvar == 3 else [u - c, u, u, u + c]
        np.testing.assert_allclose(L @ A @ R, np.diag(lam), atol=1e-7)


@pytest.mark.parametrize("flux", ["LLF", "ROE", "HLLC"])
def test_riemann_flux_consistency(flux):
    """Eq. 6: the approximate Riemann flux of two equal states is the physical flux, and a
    stationary contact (equal u = 0 and p, different rho) carries no mass (HLLC, Roe)."""
    rng = np.random.default_rng(8)
    for nvar in (3, 4):
        for _ in range(20):
            U = inputs.prim_to_cons(rng.uniform(0.2, 2), rng.uniform(-2, 2), rng.uniform(-1, 1) if nvar == 4 else 0,
                                    rng.uniform(0.1, 2), 1.4, 1 if nvar == 3 else 2)
            np.testing.assert_allclose(oracle.riemann(U, U, nvar, flux=flux), _flux_x(U), rtol=1e-13, atol=1e-13)
    if flux != "LLF":
        UL = inputs.prim_to_cons(1.0, 0.0, None, 1.0, 1.4, 1)
        UR = inputs.prim_to_cons(0.3, 0.0, None, 1.0, 1.4, 1)
        F = oracle.riemann(UL, UR, 3, flux=flux)
        np.testing.assert_allclose(F, [0.0, 1.0, 0.0], atol=1e-14)


def _run_sod(n, **kw):
    P = inputs.sod(n)
    u, t, taken, nonph = oracle.run_to(P, P.t_end, **kw)
    return P, u, t


@pytest.mark.parametrize("flux", ["HLLC", "ROE", "LLF"])
def test_sod_conservation(flux):
    """Eq. 3 telescoping with transmissive boundaries: mass and energy are constant and the
    momentum grows at exactly (p_L - p_R) = 0.9 while the waves stay inside [0, 1]."""
    P, u, t = _run_sod(200, flux=flux)
    h = P.h[0]
    assert abs(t - 0.2) < 1e-15
    m0 = P.u0.sum(axis=(1, 2)) * h
    m1 = u.sum(axis=(1, 2)) * h
    assert abs(m1[0] - m0[0]) < 1e-13 and abs(m1[2] - m0[2]) < 1e-13
    assert abs(m1[1] - 0.9 * 0.2) < 1e-13


def test_sod_matches_exact_solution():
    """Sec. 4.2.1 (Eq. 33, rescaled to [0, 1]): the density converges to the exact Riemann
    solution in L1 (first order at the discontinuities)."""
    errs = []
    for n in (200, 400, 800):
        P, u, t = _run_sod(n)
        edges = np.linspace(0.0, 1.0, n + 1)
        exact = exact_riemann.cell_average_density((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.5, t, edges)
        errs.append(np.mean(np.abs(u[0, 0] - exact)))
    assert errs[0] < 6e-3 and errs[-1] < 2e-3, errs
    assert errs[1] < errs[0] and errs[2] < errs[1], errs


def test_exact_riemann_sod_star_state():
    """Textbook star state of the Sod problem (p* = 0.30313, u* = 0.92745)."""
    ps, us = exact_riemann.star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert abs(ps - 0.30313) < 1e-5 and abs(us - 0.92745) < 1e-5


def test_mirror_symmetry_1d():
    """Reflecting x -> -x and u -> -u maps the scheme onto itself (left/right stencils mirror)."""
    P = inputs.random_piecewise_euler_1d(96, seed=3)
    L, _ = oracle.rhs(P)
    Pm = inputs.random_piecewise_euler_1d(96, seed=3)
    um = P.u0[:, :, ::-1].copy()
    um[1] *= -1
    Pm.u0 = um
    Lm, _ = oracle.rhs(Pm)
    Lm = Lm[:, :, ::-1].copy()
    Lm[1] *= -1
    np.testing.assert_allclose(Lm, L, rtol=0, atol=1e-12 * np.abs(L).max())


def test_2d_y_uniform_equals_1d():
    """A 2D state that does not vary in y evolves like the 1D Euler equations with v = 0."""
    P1 = inputs.random_piecewise_euler_1d(64, seed=4)
    U1 = P1.u0[:, 0, :]
    ny = 12
    U2 = np.zeros((4, ny, 64))
    U2[0] = U1[0]; U2[1] = U1[1]; U2[2] = 0.0; U2[3] = U1[2]
    P2 = inputs.Problem("y", 2, 4, 64, ny, (0.0, 0.0), (1.0, ny / 64.0), (1, 0), U2, 1)
    L1, _ = oracle.rhs(P1)
    L2, _ = oracle.rhs(P2)
    for j in range(ny):
        np.testing.assert_allclose(L2[[0, 1, 3], j], L1[:, 0], rtol=0, atol=1e-13 * np.abs(L1).max())
    assert np.abs(L2[2]).max() < 1e-13 * np.abs(L1).max()


def test_2d_transpose_equivariance():
    """Swapping x <-> y together with (rho u) <-> (rho v) commutes with the RHS."""
    P = inputs.riemann2d(40, seed=1)
    L, _ = oracle.rhs(P)
    UT = P.u0.transpose(0, 2, 1)[[0, 2, 1, 3]].copy()
    PT = inputs.Problem("t", 2, 4, 40, 40, (0.0, 0.0), (1.0, 1.0), (1, 1), UT, 1)
    LT, _ = oracle.rhs(PT)
    np.testing.assert_allclose(LT.transpose(0, 2, 1)[[0, 2, 1, 3]], L, rtol=0, atol=1e-12 * np.abs(L).max())


def test_2d_periodic_conservation():
    """Periodic 2D Euler: sum_ij L_ij = 0 per component to round-off."""
    P = inputs.random_smooth_euler_2d(32, 24, seed=2)
    L, _ = oracle.rhs(P, weights="FE")
    scale = np.abs(L).sum(axis=(1, 2))
    assert np.all(np.abs(L.sum(axis=(1, 2))) < 1e-13 * scale)


def test_rhs_cells_matches_full_rhs():
    """The sampled-cell evaluation equals the whole-grid evaluation bit for bit."""
    P = inputs.riemann2d(48, seed=2)
    L, _ = oracle.rhs(P)
    cells = np.array([0, 5, 47, 48 * 10 + 7, 48 * 48 - 1])
    Ls = oracle.rhs_cells(P, P.u0, cells)
    flat = L.reshape(4, -1)
    np.testing.assert_array_equal(Ls, flat[:, cells].T)


# ---------------------------------------------------------------------------
# Tangent (forward-mode) pinned by central finite differences
# ---------------------------------------------------------------------------
# The tangent checks use the Z exponent p = 2, for which tau^2 = (IS_0 - IS_2)^2 has no
# kink, so the map is analytic and a fourth-order central difference converges.  On the
# isentropic vortex the characteristic shear field is constant to ~1e-11 in the far
# field (IS_k ~ 1e-24 there); with eps = 1e-40 the Z weights then change at the 1e-12
# scale and no finite difference converges, although the tangent exists.  That case
# is checked component-wise.
JVP_CASES = [
    ("smooth2d-characteristic", lambda: inputs.random_smooth_euler_2d(16, 16, seed=1), dict(characteristic=True)),
    ("vortex-componentwise", lambda: inputs.vortex(24, seed=1), dict(characteristic=False)),
]
JVP_PARAMS = dict(weights="FE", xi=100.0, flux="LLF_FROZEN", alpha=(3.0, 3.0), zp=2)


def _fd4(f, e):
    return (-f(2 * e) + 8 * f(e) - 8 * f(-e) + f(-2 * e)) / (12 * e)


@pytest.mark.parametrize("name,make,extra", JVP_CASES)
def test_rhs_jvp_matches_central_differences(name, make, extra):
    P = make()
    params = dict(JVP_PARAMS, **extra)
    du = np.random.default_rng(11).normal(size=P.u0.shape)
    _, dL = oracle.rhs_jvp(P, P.u0, du, **params)
    fd = _fd4(lambda e: oracle.rhs(P, P.u0 + e * du, **params)[0], 1e-8)
    assert np.linalg.norm(fd - dL) < 1e-6 * np.linalg.norm(dL)


@pytest.mark.parametrize("name,make,extra", JVP_CASES)
def test_step_jvp_matches_central_differences(name, make, extra):
    P = make()
    params = dict(JVP_PARAMS, **extra)
    du = np.random.default_rng(12).normal(size=P.u0.shape)
    dt, ns = 0.1 * P.h[0], 3
    _, dT = oracle.step_jvp(P, P.u0, du, dt, ns, **params)
    fd = _fd4(lambda e: oracle.step(P, P.u0 + e * du, dt=dt, nsteps=ns, **params)[0], 1e-8)
    assert np.linalg.norm(fd - dT) < 1e-6 * np.linalg.norm(dT)


def test_flop_count_scales_with_cells():
    a = oracle.count_rhs_flops(inputs.sod(64))
    b = oracle.count_rhs_flops(inputs.sod(128))
    assert a > 0 and abs(b / a - 2.0) < 0.1


def test_app_a_fe_weights_raise_the_ideal_share():
    """App. A, Tables A.1 and A.3: over a shock-tube run the FE weights sit in the bin of the
    ideal weight more often than the Z weights, for each of the three weights (the
    absolute shares depend on settings the paper does not state, so only the ordering is
    pinned).  Sod, N = 200, RK4 at CFL 0.3 (Sec. 4), statistics of every step's RHS."""
    nb = 10000
    P = inputs.sod(200)
    H = np.zeros((2, 3, nb), dtype=np.int64)
    u, t = P.u0.copy(), 0.0
    while t < 0.2 * (1 - 1e-12):
        h, _ = oracle.weight_hist(P, u, nbins=nb)
        H += h
        u, t, _, _ = oracle.step(P, u, nsteps=1, t_end=0.2, t0=t, cfl=0.3, rk4=True)
    tot = H[0, 0].sum()
    for k, d in enumerate((1 / 16, 10 / 16, 5 / 16)):
        b = int(d * nb)
        assert H[1, k, b] > 1.3 * H[0, k, b], (k, H[0, k, b] / tot, H[1, k, b] / tot)


# ---------------------------------------------------------------------------
# JS weights (Eq. 11) and M weights (Eq. 12-13), pinned in exact rational arithmetic
# ---------------------------------------------------------------------------
def _quadratic_derivatives_at_xi(nodes, vals):
    """First and second derivative at x = 0 (x_i, h = 1) of the quadratic through
    (nodes, vals), from the Lagrange form in exact fractions.  Eq. 10's f_{i,k} and
    s_{i,k} are these derivatives on the sub-stencil S_k."""
    d1 = Fraction(0)
    d2 = Fraction(0)
    for a, (xa, ya) in enumerate(zip(nodes, vals)):
        others = [xb for b, xb in enumerate(nodes) if b != a]
        den = Fraction(1)
        for xb in others:
            den *= xa - xb
        # l_a(x) = (x - o0)(x - o1) / den: l_a'(0) = -(o0 + o1) / den, l_a'' = 2 / den
        d1 += ya * Fraction(-(others[0] + others[1])) / den
        d2 += ya * Fraction(2) / den
    return d1, d2


def _js_weights_exact(v, eps, ideal=(Fraction(1, 16), Fraction(10, 16), Fraction(5, 16))):
    """Eq. 9 with the derivatives of Eq. 10 taken from the sub-stencil quadratics, then
    Eq. 11: alpha_k = d_k / (IS_k + eps)^2, normalised over k = 0..2."""
    v = [Fraction(x) for x in v]
    eps = Fraction(eps)
    alphas = []
    for k in range(3):
        nodes = [k - 2, k - 1, k]
        f, s = _quadratic_derivatives_at_xi(nodes, v[k:k + 3])
        IS = f * f + s * s
        alphas.append(ideal[k] / ((IS + eps) ** 2))
    tot = sum(alphas)
    return [a / tot for a in alphas], alphas


def _eq8_weights_exact(v, eps):
    """The garbled Eq. 8 form d_k / (IS_k^2 + eps): a plausible misreading of Eq. 11."""
    v = [Fraction(x) for x in v]
    eps = Fraction(eps)
    ideal = (Fraction(1, 16), Fraction(10, 16), Fraction(5, 16))
    alphas = []
    for k in range(3):
        f, s = _quadratic_derivatives_at_xi([k - 2, k - 1, k], v[k:k + 3])
        IS = f * f + s * s
        alphas.append(ideal[k] / (IS * IS + eps))
    tot = sum(alphas)
    return [a / tot for a in alphas]


JS_STENCILS = [
    # (values u_{i-2}..u_{i+2}, eps): a quadratic with a jump between i and i+1, a kink,
    # a step at the left end, and a smooth cubic -- each with an eps that is not
    # negligible against IS, so the place of eps in Eq. 11 matters
    ([Fraction(0), Fraction(1, 10), Fraction(2, 5), Fraction(5, 2), Fraction(18, 5)], Fraction(1, 4)),
    ([Fraction(1), Fraction(1), Fraction(1), Fraction(3, 2), Fraction(2)], Fraction(1, 100)),
    ([Fraction(3), Fraction(0), Fraction(1, 8), Fraction(1, 2), Fraction(3, 2)], Fraction(1, 10)),
    ([Fraction(-8, 10), Fraction(-1, 10), Fraction(0), Fraction(1, 10), Fraction(8, 10)], Fraction(1, 1000)),
]


@pytest.mark.parametrize("case", range(len(JS_STENCILS)))
def test_js_weights_eq11_exact(case):
    """Eq. 11 (Sec. 2): omega_k = alpha_k / sum_l alpha_l with alpha_k = d_k / (IS_k + eps)^2,
    IS_k from Eq. 9-10 -- the oracle's base weights agree with the exact rational value to
    1e-15, and differ from the Eq. 8 form d_k / (IS_k^2 + eps) on the same stencil."""
    v, eps = JS_STENCILS[case]
    want, _ = _js_weights_exact(v, eps)
    _, wz, wf, mapped = oracle.interp([float(x) for x in v], weights="JS", eps=float(eps))
    assert mapped == 0
    np.testing.assert_allclose(wz, [float(w) for w in want], rtol=0, atol=1e-15)
    np.testing.assert_array_equal(wz, wf)  # JS weights are final as they are
    other = _eq8_weights_exact(v, eps)
    assert max(abs(float(a - b)) for a, b in zip(want, other)) > 1e-3, "stencil does not tell Eq. 8 from Eq. 11"


@pytest.mark.parametrize("case", range(len(JS_STENCILS)))
def test_m_weights_eq12_13_exact(case):
    """Eq. 12-13: the M weights map the JS weights with Henrick's g_k and renormalise;
    checked against the exact rational evaluation on the Eq. 11 stencils."""
    v, eps = JS_STENCILS[case]
    js, _ = _js_weights_exact(v, eps)
    ideal = (Fraction(1, 16), Fraction(10, 16), Fraction(5, 16))
    g = [w * (d + d * d - 3 * d * w + w * w) / (d * d + (1 - 2 * d) * w) for w, d in zip(js, ideal)]
    tot = sum(g)
    want = [float(x / tot) for x in g]
    _, wz, wf, _ = oracle.interp([float(x) for x in v], weights="M", eps=float(eps))
    np.testing.assert_allclose(wz, [float(w) for w in js], rtol=0, atol=1e-15)  # base = JS
    np.testing.assert_allclose(wf, want, rtol=0, atol=1e-15)


def test_js_interpolated_value_exact():
    """Eq. 6 with the Eq. 11 weights and the Eq. 5 sub-stencil values, each sub-stencil
    value formed independently as the quadratic interpolant at x_{i+1/2}."""
    v, eps = JS_STENCILS[0]
    w, _ = _js_weights_exact(v, eps)
    q = []
    for k in range(3):
        nodes = [k - 2, k - 1, k]
        val = Fraction(0)
        for a, xa in enumerate(nodes):
            term = v[k + a]
            for b, xb in enumerate(nodes):
                if b != a:
                    term *= (Fraction(1, 2) - xb) / Fraction(xa - xb)
            val += term
        q.append(val)
    want = float(sum(wk * qk for wk, qk in zip(w, q)))
    got, _, _, _ = oracle.interp([float(x) for x in v], weights="JS", eps=float(eps))
    assert abs(got - want) <= 4e-16 * max(1.0, abs(want))


# ---------------------------------------------------------------------------
# CFL step (Sec. 4 marches at a CFL number; the hot path's rule dt = cfl / sum_d max/h_d)
# ---------------------------------------------------------------------------
def test_cfl_step_advection_c1_exact():
    """Scalar advection, speed 1, h = 0.01, CFL 0.5: dt = 0.5 * 0.01 / 1 = 0.005, so one
    CFL step ends at t = 0.005 and 400 steps reach t = 2 up to the rounding of 400 sums
    (0.005 has no exact binary form: a 401st step of round-off size may close the gap)."""
    P = inputs.advection_sine(200)
    _, t, taken, _ = oracle.step(P, dt=0.0, nsteps=1, cfl=0.5)
    assert taken == 1 and abs(t - 0.005) <= 1e-18
    _, t, taken, _ = oracle.step(P, dt=0.0, nsteps=400, cfl=0.5)
    assert taken == 400 and abs(t - 2.0) <= 400 * 2.0 ** -52 * 2.0
    _, t, taken, _ = oracle.step(P, dt=0.0, nsteps=10 ** 6, t_end=2.0, cfl=0.5)
    assert taken in (400, 401) and t == 2.0


def test_cfl_step_sod_closed_form():
    """Sod tube: the fastest initial signal is the left state's sound speed sqrt(1.4),
    so the first CFL step is cfl * h / sqrt(gamma p_L / rho_L) = 0.5 (1/N) / sqrt(1.4)."""
    n = 512
    P = inputs.sod(n)
    wx, _ = oracle.max_wave(P)
    assert abs(wx - math.sqrt(1.4)) <= 1e-15
    _, t, _, _ = oracle.step(P, dt=0.0, nsteps=1, cfl=0.5)
    want = 0.5 * (1.0 / n) / math.sqrt(1.4)
    assert abs(t - want) <= 1e-15 * want
    # CFL 0.3 (the paper's choice, Sec. 4) scales the step linearly
    _, t3, _, _ = oracle.step(P, dt=0.0, nsteps=1, cfl=0.3)
    assert abs(t3 - 0.6 * want) <= 1e-15 * want


def test_cfl_step_2d_sums_both_directions():
    """2D: dt = cfl / ((|u| + c) / hx + (|v| + c) / hy) on a uniform state with u != v and
    hx != hy (a mistake in either term or a max in place of the sum changes it)."""
    nx, ny = 48, 40
    rho, u, v, p, gamma = 1.3, 0.7, -0.2, 0.9, 1.4
    c = math.sqrt(gamma * p / rho)
    u0 = inputs.prim_to_cons(np.full((ny, nx), rho), np.full((ny, nx), u), np.full((ny, nx), v),
                             np.full((ny, nx), p), gamma, 2)
    P = inputs.Problem("uniform2d", 2, 4, nx, ny, (0.0, 0.0), (2.0, 0.5), (1, 1), u0, 1)
    hx, hy = 2.0 / nx, 0.5 / ny
    wx, wy = oracle.max_wave(P)
    assert abs(wx - (abs(u) + c)) <= 1e-15 and abs(wy - (abs(v) + c)) <= 1e-15
    _, t, _, _ = oracle.step(P, dt=0.0, nsteps=1, cfl=0.5)
    want = 0.5 / ((abs(u) + c) / hx + (abs(v) + c) / hy)
    assert abs(t - want) <= 2e-15 * want


def test_cfl_step_clipped_at_t_end():
    """t_end clips the last step so the run ends on t_end exactly and stops there (a
    uniform periodic flow keeps max(|u| + c), hence the CFL step, constant)."""
    n, rho, u, p = 256, 1.0, 0.5, 1.0
    u0 = inputs.prim_to_cons(np.full((1, n), rho), np.full((1, n), u), None, np.full((1, n), p), 1.4, 1)
    P = inputs.Problem("uniform1d", 1, 3, n, 1, (0.0, 0.0), (1.0, 1.0), (0, 0), u0, 1)
    dt0 = 0.5 * (1.0 / n) / (u + math.sqrt(1.4 * p / rho))
    t_end = 2.5 * dt0
    _, t, taken, _ = oracle.step(P, dt=0.0, nsteps=10, t_end=t_end, cfl=0.5)
    assert t == t_end and taken == 3


# ---------------------------------------------------------------------------
# App. A weight statistics: the histogram of every one-sided interpolation of one L(u)
# ---------------------------------------------------------------------------
IDEAL = (Fraction(1, 16), Fraction(10, 16), Fraction(5, 16))
# Table 1 control values between consecutive null points (kappa = 1/2, xi = 1e6)
PLATEAUS = {0: [Fraction(1, 16), Fraction(1, 6)],
            1: [Fraction(10, 16), Fraction(1, 2), Fraction(5, 6)],
            2: [Fraction(5, 16), Fraction(1, 2)]}
NULLS_EXACT = {0: [Fraction(1, 32), (Fraction(1, 16) + Fraction(1, 11)) / 2, (Fraction(1, 11) + 1) / 2],
               1: [Fraction(10, 32), (Fraction(10, 16) + Fraction(2, 3)) / 2,
                   (Fraction(2, 3) + Fraction(10, 11)) / 2, (Fraction(10, 11) + 1) / 2],
               2: [Fraction(5, 32), (Fraction(5, 16) + Fraction(1, 3)) / 2, (Fraction(1, 3) + 1) / 2]}


def _z_weights_exact(v, eps, p=1):
    """Eq. 14-15 in exact fractions: alpha_k = d_k (1 + (tau / (IS_k + eps))^p), tau = |IS_0 - IS_2|,
    with IS_k = f_k^2 + s_k^2 (Eq. 9) from the derivatives of the sub-stencil quadratics (Eq. 10)."""
    v = [Fraction(x) for x in v]
    IS = []
    for k in range(3):
        f, s = _quadratic_derivatives_at_xi([k - 2, k - 1, k], v[k:k + 3])
        IS.append(f * f + s * s)
    tau = abs(IS[0] - IS[2])
    alpha = [d * (1 + (tau / (b + eps)) ** p) for d, b in zip(IDEAL, IS)]
    tot = sum(alpha)
    return [a / tot for a in alpha]


def _staircase_exact(k, w):
    """Eq. 20 at xi = 1e6 away from its null points: the identity below the first and above
    the last null point, the Table 1 control value between two of them."""
    z = NULLS_EXACT[k]
    j = sum(w > zz for zz in z)
    return w if j in (0, len(z)) else PLATEAUS[k][j - 1]


def _periodic_line(n):
    """Dyadic values (exact in binary) on a periodic line: a quadratic, a jump of 3, a
    linear ramp, a plateau, a cubic and a kink, so that smooth, one-jump and two-jump
    stencils all occur."""
    v = []
    for j in range(n):
        if j < 10:
            x = Fraction(j, 8)
            v.append(x * x)
        elif j < 18:
            v.append(3 + Fraction(j, 16))
        elif j < 24:
            v.append(Fraction(5, 2))
        elif j < 32:
            x = Fraction(j - 28, 4)
            v.append(x * x * x / 8)
        else:
            v.append(Fraction(abs(j - 36), 2))
    return v


def test_weight_hist_brute_force_in_exact_fractions():
    """App. A statistics, pinned by brute force: on a periodic scalar line, enumerate the
    interfaces k+1/2 that Eq. 3 reads for one L(u) (k = -3..n+1, so F at i-5/2..i+5/2 exists
    for every cell), form both one-sided 5-cell stencils (the right-biased one mirrored),
    compute the Z weights of Eq. 14-15 in exact fractions and the final weights through the
    Table 1 staircase and the renormalisation, bin each into [0, 1] / nbins, and compare
    with the oracle's histograms bin for bin."""
    n, nb = 40, 10000
    vals = _periodic_line(n)
    P = inputs.advection_sine(n)
    P.u0[0, 0, :] = [float(x) for x in vals]
    assert all(Fraction(float(x)) == x for x in vals)
    eps = Fraction(1e-40)

    def binned(w):
        # floor(w nbins + 1e-6), clipped; the bin must not change within 1e-9 of the
        # exact value, far more than the oracle's rounding of w moves w nbins
        x = w * nb + Fraction(1, 10 ** 6)
        lo, hi = (min(nb - 1, math.floor(x + d)) for d in (-Fraction(1, 10 ** 9), Fraction(1, 10 ** 9)))
        assert lo == hi, "weight on a bin edge"
        return lo

    want = np.zeros((2, 3, nb), dtype=np.int64)
    samples = 0
    for k in range(-3, n + 2):
        cells = [vals[(k - 2 + s) % n] for s in range(6)]
        for stencil in (cells[0:5], cells[5:0:-1]):
            wz = _z_weights_exact(stencil, eps)
            for i in range(3):
                assert min(abs(wz[i] - zz) for zz in NULLS_EXACT[i]) > Fraction(1, 10 ** 4)
            g = [_staircase_exact(i, wz[i]) for i in range(3)]
            wf = [x / sum(g) for x in g]
            for i in range(3):
                want[0, i, binned(wz[i])] += 1
                want[1, i, binned(wf[i])] += 1
            samples += 1
    got, ns = oracle.weight_hist(P, nbins=nb)
    assert ns == samples == 2 * (n + 5)
    np.testing.assert_array_equal(got, want)
    # the data reach every kind of stencil: ideal, intermediate and near-zero weights
    assert want[1, 1, 6250] > 0 and want[1, 1, 5000] > 0 and want[0, 1, :100].sum() > 0


@pytest.mark.parametrize("ndim,family,lines", [(1, "WCNS", (64,)), (2, "WCNS", (24, 16)),
                                                (1, "WENO", (64,)), (2, "WENO", (24, 16))])
def test_weight_hist_sample_counts(ndim, family, lines):
    """Every one-sided interpolation of one L(u) is counted once: Eq. 3 reads n + 5
    interfaces per line (F at i-5/2..i+5/2 for i = 0..n-1), the two-point difference of
    App. B n + 1; each interface has two one-sided interpolations per characteristic field
    (left and right states, or the f+ and f- halves of the split flux), and each histogram
    row sums to the sample count."""
    if ndim == 1:
        P = inputs.sod(lines[0])
        per = lambda m: m + (5 if family == "WCNS" else 1)
        want = 2 * P.nvar * per(P.nx)
    else:
        P = inputs.riemann2d(lines[0], seed=0, ny=lines[1])
        per = lambda m: m + (5 if family == "WCNS" else 1)
        want = 2 * P.nvar * (P.ny * per(P.nx) + P.nx * per(P.ny))
    h, ns = oracle.weight_hist(P, nbins=1000, family=family)
    assert ns == want
    assert np.all(h.sum(axis=2) == ns)


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("case", range(len(JS_STENCILS)))
def test_z_weights_eq14_15_exact(case, p):
    """Eq. 14-15: the oracle's Z weights agree with the exact rational value on the Eq. 11
    stencils (eps comparable with IS, so its place in Eq. 14 matters), for p = 1 and 2;
    with the FE map off they are also the final weights."""
    v, eps = JS_STENCILS[case]
    want = _z_weights_exact(v, eps, p=p)
    _, wz, wf, mapped = oracle.interp([float(x) for x in v], weights="Z", eps=float(eps), zp=p)
    assert mapped == 0
    np.testing.assert_allclose(wz, [float(w) for w in want], rtol=0, atol=1e-15)
    np.testing.assert_array_equal(wz, wf)


@pytest.mark.parametrize("params", [dict(), dict(weights="JS", flux="ROE"), dict(weights="M", flux="LLF"),
                                    dict(characteristic=False, zp=2), dict(family="WENO")])
def test_periodic_shift_equivariance(params):
    """On a periodic grid the scheme is translation invariant: L(shift(u)) = shift(L(u)) bit
    for bit, for shifts across the wrap in both directions (the ghost cells of Eq. 3's
    stencils come from the other end of the line, so a wrap-around index error breaks it)."""
    P = inputs.rough_euler_2d(24, 20, seed=3)
    L, _ = oracle.rhs(P, **params)
    for sx, sy in ((1, 0), (0, 1), (5, -3), (-7, 11)):
        Q = inputs.Problem("shifted", 2, 4, P.nx, P.ny, P.lo, P.hi, P.bc,
                           np.roll(P.u0, (sy, sx), axis=(1, 2)).copy(), 1)
        Ls, _ = oracle.rhs(Q, **params)
        np.testing.assert_array_equal(Ls, np.roll(L, (sy, sx), axis=(1, 2)))
    P1 = inputs.random_smooth_euler_1d(37, seed=2)
    L1, _ = oracle.rhs(P1, **params)
    for s in (1, -4, 18):
        Q1 = inputs.Problem("shifted1d", 1, 3, P1.nx, 1, P1.lo, P1.hi, P1.bc,
                            np.roll(P1.u0, s, axis=2).copy(), 1)
        np.testing.assert_array_equal(oracle.rhs(Q1, **params)[0], np.roll(L1, s, axis=2))
