"""Pins of the oracle's FE-WENO family (App. B): the fifth-order finite-difference WENO
reconstruction on Lax-Friedrichs split fluxes with the FE map of Table B.2.

Each check is independent of the oracle's own formulas: control values printed in
Table B.1, candidate polynomials rebuilt from cell averages by a linear solve, the
Jiang-Shu indicators from their integral definition, conservation, the exact Riemann
solution and the order of accuracy.
"""
from fractions import Fraction
import os

import numpy as np
import pytest

import oracle
from oracle import exact_riemann
from paper_2306_09760_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
WENO = dict(family="WENO")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [l.split() for l in f if l.strip() and not l.startswith("#")]


def test_tableB1_control_values_at_large_xi():
    """Table B.1: the App. B map sends every control point to its control value."""
    for case, i, orig, mapped in _rows("tableB1_control_values.txt"):
        g = oracle.fe_map_weno(int(i), float(Fraction(orig)), xi=1e6, kappa=0.5)
        assert abs(g - float(Fraction(mapped))) <= 1e-15, (case, i, orig, g)
    for i in range(3):
        assert oracle.fe_map_weno(i, 0.0) == 0.0


# --- polynomials with prescribed cell averages on unit cells -------------------------
def _avg_poly(cells, avgs):
    """Coefficients (lowest first) of the polynomial of degree len(cells) - 1 whose averages
    over the unit cells [c - 1/2, c + 1/2] (c in `cells`) are `avgs`."""
    n = len(cells)
    A = np.zeros((n, n))
    for r, c in enumerate(cells):
        for p in range(n):
            A[r, p] = ((c + 0.5) ** (p + 1) - (c - 0.5) ** (p + 1)) / (p + 1)
    return np.linalg.solve(A, np.asarray(avgs, dtype=np.float64))


def _peval(coef, x):
    return sum(a * x ** p for p, a in enumerate(coef))


def _pderiv(coef):
    return [p * a for p, a in enumerate(coef)][1:]


def _pint_sq(coef, a, b):
    """Integral of p(x)^2 over [a, b]."""
    sq = np.convolve(coef, coef)
    return sum(c * (b ** (p + 1) - a ** (p + 1)) / (p + 1) for p, c in enumerate(sq))


def _candidate(v, k):
    """Quadratic of sub-stencil S_k (cells k-2..k, i.e. v[k..k+2] at cells -2+k..k)."""
    cells = [-2 + k, -1 + k, k]
    return _avg_poly(cells, v[k:k + 3])


def test_ideal_combination_is_the_cell_average_quartic():
    """With JS weights and a huge eps the weights are the ideal (1/10, 6/10, 3/10) and the
    value at x_{i+1/2} is the quartic through the five cell averages."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        v = rng.normal(size=5)
        r, _, wf, _ = oracle.interp(v, weights="JS", eps=1e30, **WENO)
        np.testing.assert_allclose(wf, [0.1, 0.6, 0.3], rtol=0, atol=1e-15)
        expect = _peval(_avg_poly([-2, -1, 0, 1, 2], v), 0.5)
        assert abs(r - expect) < 1e-13 * (1 + np.abs(v).max()), (r, expect)


@pytest.mark.parametrize("case,k", [("Case3", 0), ("Case2", 2)])
def test_single_candidate_cases(case, k):
    """Table B.1 Case3 (weight 1 on S0) and Case2 (weight 1 on S2): the value is that
    sub-stencil's quadratic at x_{i+1/2}."""
    x = np.arange(-2, 3, dtype=np.float64)
    v = 0.3 * x + 0.05 * x ** 2
    if case == "Case3":
        v[3:] += 1e6      # jump between x_i and x_{i+1}
    else:
        v[:2] += 1e6      # jump between x_{i-1} and x_i
    r, _, wf, _ = oracle.interp(v, weights="FE", **WENO)
    assert abs(wf[k] - 1.0) < 1e-12
    expect = _peval(_candidate(v, k), 0.5)
    assert abs(r - expect) < 1e-9 * np.abs(v).max(), (r, expect)


def _jiang_shu(v, k):
    """beta_k = sum_{l=1,2} int_{-1/2}^{1/2} (d^l p_k / dx^l)^2 dx on unit cells."""
    p = _candidate(v, k)
    d1 = _pderiv(p)
    d2 = _pderiv(d1)
    return _pint_sq(d1, -0.5, 0.5) + _pint_sq(d2, -0.5, 0.5)


def test_indicators_match_the_integral_definition():
    """The Z weights (Eq. 14-15, p = 1) built from the integral-defined indicators equal the
    oracle's base weights of the WENO family."""
    rng = np.random.default_rng(12)
    d = np.array([0.1, 0.6, 0.3])
    for _ in range(50):
        v = rng.normal(size=5)
        beta = np.array([_jiang_shu(v, k) for k in range(3)])
        tau = abs(beta[0] - beta[2])
        a = d * (1 + tau / (beta + 1e-40))
        _, wz, _, _ = oracle.interp(v, weights="Z", **WENO)
        np.testing.assert_allclose(wz, a / a.sum(), rtol=1e-12, atol=1e-15)


def test_embedded_cases_1_and_4():
    """Table B.1: a jump in S0 only gives original weights (0, 2/3, 1/3) mapped to
    (0, 1/2, 1/2); a jump in S2 only gives (1/7, 6/7, 0) mapped to (1/4, 3/4, 0)."""
    x = np.arange(-2, 3, dtype=np.float64)
    v = 0.1 * x
    v1 = v.copy(); v1[0] += 1e6
    _, wz, wf, _ = oracle.interp(v1, weights="FE", **WENO)
    np.testing.assert_allclose(wz, [0, 2 / 3, 1 / 3], atol=1e-5)
    np.testing.assert_allclose(wf, [0, 0.5, 0.5], atol=1e-12)
    v4 = v.copy(); v4[4] += 1e6
    _, wz, wf, _ = oracle.interp(v4, weights="FE", **WENO)
    np.testing.assert_allclose(wz, [1 / 7, 6 / 7, 0], atol=1e-5)
    np.testing.assert_allclose(wf, [0.25, 0.75, 0], atol=1e-12)


@pytest.mark.parametrize("characteristic", [True, False])
def test_split_flux_is_consistent(characteristic):
    """f+ + f- = f: on six equal states the interface flux is the physical flux, with or
    without the characteristic projection (L R = I)."""
    rho, u, v, p = 0.8, 0.3, -0.2, 1.1
    E = p / 0.4 + 0.5 * rho * (u * u + v * v)
    U = np.array([rho, rho * u, rho * v, E])
    F, fb = oracle.interface_flux(np.tile(U, (6, 1)), 4, characteristic=characteristic, **WENO)
    expect = [rho * u, rho * u * u + p, rho * u * v, (E + p) * u]
    np.testing.assert_allclose(F, expect, rtol=1e-13)
    assert not fb


def test_order_five_on_smooth_advection():
    errs = []
    for n in (40, 80, 160, 320):
        x = -1.0 + np.arange(n) * (2.0 / n)
        P = inputs.Problem("adv", 1, 1, n, 1, (0.0, 0.0), (2.0, 1.0), (0, 0),
                           np.sin(np.pi * x)[None, None, :].copy(), 0, adv_speed=(1.0, 0.0))
        L, _ = oracle.rhs(P, **WENO)
        errs.append(np.max(np.abs(L[0, 0] + np.pi * np.cos(np.pi * x))))
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(order > 4.8) and np.all(order < 5.3), order


def test_periodic_conservation():
    """Conservative difference: sum_i L_i = 0 to round-off on a periodic Euler line."""
    P = inputs.random_piecewise_euler_1d(300, seed=3)
    P = inputs.Problem(P.name, 1, 3, P.nx, 1, P.lo, P.hi, (0, 0), P.u0, 1)
    L, _ = oracle.rhs(P, **WENO)
    scale = np.abs(L).max()
    assert np.all(np.abs(L.sum(axis=(1, 2))) < 1e-12 * scale * P.nx)


def test_sod_matches_exact_solution():
    errs = []
    for n in (200, 400, 800):
        P = inputs.sod(n)
        u, t, _, _ = oracle.run_to(P, P.t_end, **WENO)
        edges = np.linspace(0.0, 1.0, n + 1)
        exact = exact_riemann.cell_average_density((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.5, t, edges)
        errs.append(np.mean(np.abs(u[0, 0] - exact)))
    assert errs[0] < 6e-3 and errs[-1] < 2e-3, errs
    assert errs[1] < errs[0] and errs[2] < errs[1], errs
