"""Pins of the oracle's boundary faces (Sec. 4.3): inviscid wall, fixed inflow state and
the moving oblique shock of the double Mach reflection."""
import numpy as np
import pytest

import oracle
from paper_2306_09760_gb300 import inputs

WALL, FIXED, TRANS = inputs.FACE_WALL, inputs.FACE_FIXED, inputs.FACE_TRANSMISSIVE


def _smooth_2d(nx, ny, seed, ylo=0.0, yhi=1.0, bc=(1, 1)):
    P = inputs.random_smooth_euler_2d(nx, ny, seed=seed)
    return inputs.Problem("s", 2, 4, nx, ny, (0.0, ylo), (1.0, yhi), bc, P.u0.copy(), 1)


@pytest.mark.parametrize("family", ["WCNS", "WENO"])
def test_wall_equals_mirrored_domain(family):
    """A wall at y = 0 gives the same L as the domain doubled by mirroring (rho, rho u, E
    even, rho v odd) with the mirror image as real cells."""
    nx, ny = 24, 16
    P = _smooth_2d(nx, ny, seed=7)
    P.extra = {"faces": {"types": (TRANS, TRANS, WALL, TRANS)}}
    L, _ = oracle.rhs(P, family=family)
    m = P.u0[:, ::-1, :].copy()
    m[2] *= -1.0
    D = inputs.Problem("d", 2, 4, nx, 2 * ny, (0.0, -1.0), (1.0, 1.0), (1, 1),
                       np.concatenate([m, P.u0], axis=1), 1)
    Ld, _ = oracle.rhs(D, family=family)
    np.testing.assert_array_equal(L, Ld[:, ny:, :])


def test_walls_conserve_mass_and_energy():
    """Walls on both y faces, periodic x: no mass or energy crosses the boundary."""
    P = _smooth_2d(32, 20, seed=3, bc=(0, 1))
    P.extra = {"faces": {"types": (0, 0, WALL, WALL)}}
    u, _, _, _ = oracle.step(P, nsteps=10)
    s0, s1 = P.u0.sum(axis=(1, 2)), u.sum(axis=(1, 2))
    for k in (0, 3):
        assert abs(s1[k] - s0[k]) < 1e-12 * abs(s0[k]), (k, s1[k] - s0[k])


def test_fixed_face_with_its_own_state_is_steady():
    state = (1.3, 0.4, -0.2, 0.9)
    nx, ny = 20, 12
    rho, u, v, p = (np.full((ny, nx), a) for a in state)
    u0 = inputs.prim_to_cons(rho, u, v, p, 1.4, 2)
    P = inputs.Problem("f", 2, 4, nx, ny, (0.0, 0.0), (1.0, 1.0), (1, 1), u0, 1,
                       extra={"faces": {"types": (FIXED, FIXED, FIXED, FIXED), "state_a": state}})
    L, _ = oracle.rhs(P)
    assert np.all(L == 0.0)


def test_dmr_shock_moves_at_the_exact_speed():
    """Sec. 4.3: along the top boundary the Mach 10 shock (normal speed 10 into gas with
    c = 1) moves at 20/sqrt(3) in x; at t = 0.2 the density jump in the top row sits at
    1/6 + (1 + 20 t)/sqrt(3) (FE-WENO family, 240 x 60 cells)."""
    P = inputs.dmr(240, 60)
    u, t, _, nonph = oracle.run_to(P, 0.2, family="WENO")
    assert t == 0.2 and nonph == 0
    rho_top = u[0, -1, :]
    x = (np.arange(240) + 0.5) * (4.0 / 240)
    front = x[np.argmax(rho_top < 0.5 * (8.0 + 1.4))]
    exact = 1.0 / 6.0 + (1.0 + 20.0 * 0.2) / np.sqrt(3.0)
    assert abs(front - exact) < 3 * (4.0 / 240), (front, exact)


def test_eq3_difference_loses_positivity_at_the_dmr_shock():
    """Why the double Mach reflection (Sec. 4.3) runs with the FE-WENO family: across the
    Mach 10 shock (pressure ratio 116.5) the sixth-order midpoint difference of Eq. 3,
    whose second and third coefficients reach two and three interfaces upstream with
    d2 < 0, drives the second pre-shock cell to a negative pressure in the first RK
    stage at CFL 0.5 -- with the very interface fluxes under which the two-point
    difference of App. B keeps every cell physical.  (The 2D problem fails the same way
    on every row at the shock front, not only next to the wall.)"""
    g, n = 1.4, 400
    x = inputs.cell_centres(0.0, 1.0, n)
    post, pre = (8.0, 8.25, 116.5), (1.4, 0.0, 1.0)  # normal-shock states of the DMR
    prim = [np.where(x < 0.3, a, b) for a, b in zip(post, pre)]
    u0 = inputs.prim_to_cons(prim[0][None, :], prim[1][None, :], None, prim[2][None, :], g, 1)
    U = u0[:, 0, :].T

    def cell(k):
        return U[min(max(k, 0), n - 1)]

    # F[k + 3] = F_{k+1/2}, the WCNS-FE interface flux (characteristic FE, HLLC)
    F = np.array([oracle.interface_flux(np.array([cell(k + m) for m in range(-2, 4)]), 3)[0]
                  for k in range(-3, n + 2)])
    h = 1.0 / n
    dt = 0.5 * h / (8.25 + np.sqrt(g * 116.5 / 8.0))
    d1, d2, d3 = 75 / 64, -25 / 384, 3 / 640
    bad_eq3, bad_two_point = [], []
    for i in range(n):
        f = [F[i + 3 + m] for m in range(-3, 3)]  # F_{i-5/2} .. F_{i+5/2}
        L3 = -(d1 * (f[3] - f[2]) + d2 * (f[4] - f[1]) + d3 * (f[5] - f[0])) / h
        L2 = -(f[3] - f[2]) / h
        for L, bad in ((L3, bad_eq3), (L2, bad_two_point)):
            v = U[i] + dt * L
            if not (v[0] > 0 and (g - 1) * (v[2] - 0.5 * v[1] ** 2 / v[0]) > 0):
                bad.append(i)
    first_pre = int(np.argmax(x >= 0.3))
    assert bad_eq3 == [first_pre + 1]
    assert bad_two_point == []
