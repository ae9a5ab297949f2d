"""The single-precision path across the weight, flux and projection options, and at the
limits of single precision.

In single precision eps = 1e-40 is subnormal (and flushed to zero), so the kernels raise
it to 2^-126 and cap the Z ratio tau / (IS + eps) of Eq. 15 at 1e18.  Two inputs reach
those limits: exactly constant data (every IS is 0, so the ratio would be 0 / 0) and a
jump next to constant cells (IS of the smooth stencil is 0 while tau is large, so the
ratio would overflow).  In both cases the weights must reach the limits the
double-precision oracle reaches, with no interface falling back to first order.
"""
import numpy as np
import pytest

import oracle
from paper_2306_09760_gb300 import inputs

pytestmark = pytest.mark.gpu

WEIGHTS = ["JS", "Z", "FE", "PFE", "M"]


def weight_params(weights):
    # JS and M square IS + eps, so in single precision eps must keep eps^2 normal
    return dict(weights=weights, eps=1e-6) if weights in ("JS", "M") else dict(weights=weights)


@pytest.fixture(scope="module")
def W():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2306_09760_gb300 import build as wbuild
    wbuild.build()
    from paper_2306_09760_gb300 import wcns
    wcns.load()
    return wcns


@pytest.fixture(scope="module")
def stream(W):
    import torch
    return torch.cuda.Stream()


def gpu_rhs32(W, stream, P, **params):
    import torch
    with torch.cuda.stream(stream):
        S = W.Solver(P, "f32", stream=stream, **params)
        L = S.numpy(S.rhs())
        st, nonph = S.status()
        S.close()
    assert st == W.WCNS_OK, W.wcns_status_string(st)
    return L.astype(np.float64), nonph


def constant_problem(ndim, bc):
    """rho = 1, u = 0.5, v = 0.25, p = 1: every conserved value and every product in the
    projection is a short binary fraction, so stencils are exactly constant."""
    if ndim == 1:
        u0 = inputs.prim_to_cons(np.ones((1, 300)), np.full((1, 300), 0.5), None, np.ones((1, 300)), 1.4, 1)
        return inputs.Problem("const1d", 1, 3, 300, 1, (0.0, 0.0), (1.0, 1.0), (bc, bc), u0, 1)
    shape = (37, 40)
    u0 = inputs.prim_to_cons(np.ones(shape), np.full(shape, 0.5), np.full(shape, 0.25), np.ones(shape), 1.4, 2)
    return inputs.Problem("const2d", 2, 4, 40, 37, (0.0, 0.0), (1.0, 1.0), (bc, bc), u0, 1)


def jump_problem(n=700):
    """A strong 1D jump (rho 1 -> 10, p 1 -> 100, u = 0) with constant states on both sides."""
    x = (np.arange(n) + 0.5) / n
    rho = np.where(x < 0.43, 1.0, 10.0)[None, :]
    p = np.where(x < 0.43, 1.0, 100.0)[None, :]
    u0 = inputs.prim_to_cons(rho, np.zeros_like(rho), None, p, 1.4, 1)
    return inputs.Problem("jump", 1, 3, n, 1, (0.0, 0.0), (1.0, 1.0), (1, 1), u0, 1)


@pytest.mark.parametrize("weights", WEIGHTS)
@pytest.mark.parametrize("flux", ["LLF", "ROE", "HLLC"])
@pytest.mark.parametrize("characteristic", [True, False])
def test_f32_option_matrix(W, stream, weights, flux, characteristic):
    params = dict(flux=flux, characteristic=characteristic, **weight_params(weights))
    for Q in (inputs.random_piecewise_euler_1d(700, seed=5), inputs.riemann2d(70, seed=2, ny=66)):
        L, nonph = gpu_rhs32(W, stream, Q, **params)
        Lr, nonph_r = oracle.rhs(Q, **params)
        err = np.abs(L - Lr)
        rel_l1 = err.mean() / np.abs(Lr).mean()
        assert rel_l1 < 1e-4, (Q.name, rel_l1)
        # per element: a misplaced cell or ghost would show as an O(|L|) error
        assert err.max() < 3e-3 * np.abs(Lr).max(), (Q.name, err.max() / np.abs(Lr).max())
        assert nonph == nonph_r == 0, (Q.name, nonph, nonph_r)


@pytest.mark.parametrize("weights", WEIGHTS)
@pytest.mark.parametrize("characteristic", [True, False])
@pytest.mark.parametrize("ndim,bc", [(1, 0), (1, 1), (2, 0), (2, 1)])
def test_f32_exactly_constant_state(W, stream, weights, characteristic, ndim, bc):
    """Every IS is exactly 0: L must be exactly 0 and no interface may fall back."""
    P = constant_problem(ndim, bc)
    L, nonph = gpu_rhs32(W, stream, P, characteristic=characteristic, **weight_params(weights))
    assert nonph == 0
    assert np.all(L == 0.0), float(np.max(np.abs(L)))


@pytest.mark.parametrize("weights", ["Z", "FE", "PFE"])
@pytest.mark.parametrize("characteristic", [True, False])
def test_f32_jump_next_to_constant_state(W, stream, weights, characteristic):
    """IS of the smooth stencil is exactly 0 next to the jump while tau ~ 1e4: the capped
    ratio must give the oracle's weights (the smooth stencil takes the whole weight)."""
    P = jump_problem()
    params = dict(weights=weights, characteristic=characteristic)
    L, nonph = gpu_rhs32(W, stream, P, **params)
    Lr, nonph_r = oracle.rhs(P, **params)
    assert nonph == nonph_r == 0
    err = np.max(np.abs(L - Lr)) / np.max(np.abs(Lr))
    assert err < 1e-4, err
