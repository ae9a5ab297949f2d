"""Parity at the full 2D size (2048 x 2048, four-quadrant Riemann data) on sampled cells.

The oracle evaluates L at chosen cells directly; a full TVD-RK3 step at an interior
cell depends only on the 31 x 31 patch around it (three stages of radius 5), so the
oracle steps that patch and the centre value is exact.  The same launch configuration
as the benchmark is used (2D x sweep + fused y sweep/stage kernels).
"""
import numpy as np
import pytest

import oracle
from paper_2306_09760_gb300 import inputs

pytestmark = pytest.mark.gpu

N = 2048


@pytest.fixture(scope="module")
def W():
    import torch
    assert torch.cuda.is_available()
    from paper_2306_09760_gb300 import build as wbuild
    wbuild.build()
    from paper_2306_09760_gb300 import wcns
    return wcns


@pytest.fixture(scope="module")
def problem():
    return inputs.riemann2d(N, seed=0)


def sample_cells(n, rng, count, margin=0):
    """Random cells plus cells on the quadrant lines (x, y = 0.8) and near the edges."""
    i = rng.integers(margin, n - margin, count)
    j = rng.integers(margin, n - margin, count)
    k = int(0.8 * n)
    extra_i = np.concatenate([np.full(40, k - 1), np.full(40, k), rng.integers(margin, n - margin, 80)])
    extra_j = np.concatenate([rng.integers(margin, n - margin, 80), np.full(40, k - 1), np.full(40, k)])
    if margin == 0:
        extra_i = np.concatenate([extra_i, [0, 1, 2, n - 1, n - 3, 0, n - 1]])
        extra_j = np.concatenate([extra_j, [5, 0, n - 1, 7, n - 2, 0, n - 1]])
    return np.concatenate([i, extra_i]), np.concatenate([j, extra_j])


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_fullsize_rhs_sampled(W, problem, dtype):
    import torch
    P = problem
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        S = W.Solver(P, dtype, stream=stream)
        L = S.rhs()
        torch.cuda.synchronize()
        rng = np.random.default_rng(0)
        ii, jj = sample_cells(N, rng, 3000)
        got = L[:, torch.as_tensor(jj, device="cuda"), torch.as_tensor(ii, device="cuda")].double().cpu().numpy().T
        S.close()
    ref = oracle.rhs_cells(P, P.u0, jj * N + ii)
    if dtype == "f64":
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        if err >= 1e-11:
            from parity import perturb_ulp
            sens = np.max(np.abs(oracle.rhs_cells(P, perturb_ulp(P.u0), jj * N + ii) - ref)) / np.max(np.abs(ref))
            assert err < 10 * sens, (err, sens)
    else:
        err = np.abs(got - ref).mean() / np.abs(ref).mean()
        assert err < 1e-4, err


def test_fullsize_step_sampled(W, problem):
    import torch
    P = problem
    wx, wy = oracle.max_wave(P)
    dt = 0.5 / (wx / P.h[0] + wy / P.h[1])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        S = W.Solver(P, "f64", stream=stream)
        S.step(dt, 1)
        torch.cuda.synchronize()
        rng = np.random.default_rng(1)
        ii, jj = sample_cells(N, rng, 150, margin=16)
        got = S.u[:, torch.as_tensor(jj, device="cuda"), torch.as_tensor(ii, device="cuda")].cpu().numpy().T
        st, _ = S.status()
        S.close()
    assert st == W.WCNS_OK
    ref = np.zeros_like(got)
    for s, (i, j) in enumerate(zip(ii, jj)):
        patch = P.u0[:, j - 15:j + 16, i - 15:i + 16].copy()
        Q = inputs.Problem("patch", 2, 4, 31, 31, (0.0, 0.0), (31 * P.h[0], 31 * P.h[1]), (1, 1), patch, 1)
        u, _, _, _ = oracle.step(Q, dt=dt, nsteps=1)
        ref[s] = u[:, 15, 15]
    err = np.max(np.abs(got - ref)) / np.max(np.abs(P.u0))
    assert err < 1e-11, err
