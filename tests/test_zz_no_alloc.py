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
