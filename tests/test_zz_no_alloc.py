"""The allocation-free reduction entry point (wcns_reduce_noalloc).

Some callers cannot allocate device memory where they need a sum or a norm (their
memory is reserved up front, or another allocator owns it), so they cannot create a
context either.  This checks, through the C ABI, that the context-free entry point --
whose scratch is a fixed static device array -- returns what wcns_reduce returns, on two
calls in a row (the second call reuses the array the first one left behind).  The file
is named to be collected last.
"""
import numpy as np
import pytest

from paper_2306_09760_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import torch
    assert torch.cuda.is_available()
    from paper_2306_09760_gb300 import build as wbuild
    wbuild.build()
    from paper_2306_09760_gb300 import wcns
    return wcns


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_reduce_matches_context_reduce(W, dtype):
    import torch
    P = inputs.riemann2d(700, seed=4, ny=333)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        S = W.Solver(P, dtype, stream=stream)
        other = S.alloc()
        S.set_state(P.u0 * 0.75 + 0.01, other)
        out = torch.zeros(8, dtype=torch.float64, device="cuda")
        for what in (W.WCNS_REDUCE_SUM, W.WCNS_REDUCE_L1, W.WCNS_REDUCE_LINF):
            for b in (None, other):
                ref = W.wcns_reduce(S.ctx, S.u, b, what, S.grid.nvar)
                for call in range(2):
                    out.fill_(-1.0)
                    W.wcns_reduce_noalloc(S.grid, S.u, b, what, out, stream)
                    stream.synchronize()
                    got = out[: S.grid.nvar].cpu().numpy()
                    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=0,
                                               err_msg=f"what={what} b={'set' if b is not None else 'none'} call={call}")
        S.close()


def test_noalloc_reduce_rejects_too_many_variables(W):
    g = W.wcns_grid()
    g.ndim, g.nvar, g.dtype, g.nx, g.ny, g.pitch = 1, 5, 0, 64, 1, 64
    with pytest.raises(W.WcnsError) as e:
        W.wcns_reduce_noalloc(g, 16, None, W.WCNS_REDUCE_SUM, 16)
    assert e.value.status == W.WCNS_ERR_ARG


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_noalloc_reduce_fills_the_whole_array(W, dtype):
    """2048 x 1024 cells per plane and four planes: the grid asks for 2048 blocks per
    variable, is clamped to the 2040 the array holds, and so writes the last row of
    partials.  The context path uses another block count, hence a tolerance."""
    import torch
    P = inputs.riemann2d(2048, seed=1, ny=1024)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        S = W.Solver(P, dtype, stream=stream)
        assert S.grid.nvar == 4
        other = S.alloc()
        S.set_state(P.u0 * 1.25 - 0.02, other)
        out = torch.zeros(4, dtype=torch.float64, device="cuda")
        for what in (W.WCNS_REDUCE_SUM, W.WCNS_REDUCE_L1, W.WCNS_REDUCE_LINF):
            ref = W.wcns_reduce(S.ctx, S.u, other, what, 4)
            for call in range(2):
                out.fill_(-1.0)
                W.wcns_reduce_noalloc(S.grid, S.u, other, what, out, stream)
                stream.synchronize()
                np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=0,
                                           err_msg=f"what={what} call={call}")
        S.close()


def test_noalloc_reduce_independent_lines(W):
    """ndim = 1 with ny > 1 (independent lines), accepted as wcns_init accepts it."""
    import torch
    rng = np.random.default_rng(3)
    nx, ny, pitch = 300, 7, 320
    host = np.zeros((3, ny, pitch))
    host[:, :, :nx] = rng.uniform(-1.0, 2.0, size=(3, ny, nx))
    a = torch.from_numpy(host).cuda()
    g = W.wcns_grid()
    g.ndim, g.nvar, g.dtype, g.nx, g.ny, g.pitch = 1, 3, 0, nx, ny, pitch
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    W.wcns_reduce_noalloc(g, a, None, W.WCNS_REDUCE_SUM, out, None)
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), host[:, :, :nx].sum(axis=(1, 2)), rtol=1e-13)
    W.wcns_reduce_noalloc(g, a, None, W.WCNS_REDUCE_LINF, out, None)
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), np.abs(host[:, :, :nx]).max(axis=(1, 2)), rtol=0)
