"""The banded 2D stage against the two-launch stage.

On 2D Euler grids of more than four bands of rows each RK stage runs as one persistent
launch: the x-direction interfaces of a band of rows write the band's partial stage into
a ring slot, and the band's y-direction interfaces complete the stage from it.  It
evaluates the same interface fluxes (Eq. 6), Eq. 3 differences and stage updates with the
same arithmetic as the x-sweep and y-sweep launches over the whole grid, so the two forms
must give the same states bit for bit, the same device time and the same fallback counts
-- at band edges, the ragged last band and x tile, both boundary kinds, single and
double precision, TVD-RK3 and the Eq. 16 stages, graph replay and direct launches, and a
run that stops at t_end.  The two-launch form is the one the oracle parity tests cover.
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


def _run(W, P, dtype, banded, calls, params):
    import torch
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        S = W.Solver(P, dtype, stream=stream, **params)
        W.wcns_set_stage_form(S.ctx, banded)
        for dt, n, t_end in calls:
            S.step(dt, n, t_end)
        stream.synchronize()
        u = S.u.clone()
        t, steps = S.time()
        st, fb = S.status()
        S.close()
    return u, t, steps, st, fb


CASES = {
    # 2048 x 700 FP32, default scheme: ragged x tile (10 cells) and ragged last band (100 rows)
    "riemann_2048x700_f32": (lambda: inputs.riemann2d(2048, seed=2, ny=700), "f32", {},
                             [(0.0, 1, 0.0), (0.0, 3, 0.0)]),
    # periodic smooth data, 1300 x 1000: two x tiles (1019 and 281 cells), seven bands
    "smooth_1300x1000_f32": (lambda: inputs.random_smooth_euler_2d(1300, 1000, seed=3), "f32", {},
                             [(0.0, 2, 0.0), (0.0, 1, 0.0)]),
    # the Eq. 16 stages (general stage form)
    "riemann_2048x700_f32_rk4": (lambda: inputs.riemann2d(2048, seed=5, ny=700), "f32", {"integrator": "RK4"},
                                 [(0.0, 2, 0.0)]),
    # a run that reaches t_end inside the call: the later steps change nothing
    "riemann_2048x640_f32_tend": (lambda: inputs.riemann2d(2048, seed=6, ny=640), "f32", {},
                                  [(2.0e-4, 1, 5.0e-4), (2.0e-4, 4, 5.0e-4)]),
    # FP64: one-interface x tiles (251 cells), six bands
    "riemann_700x900_f64": (lambda: inputs.riemann2d(700, seed=1, ny=900), "f64", {}, [(0.0, 2, 0.0)]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_banded_stage_equals_two_launch_stage(W, name):
    make, dtype, params, calls = CASES[name]
    P = make()
    ub, tb, nb, stb, fbb = _run(W, P, dtype, True, calls, params)
    u2, t2, n2, st2, fb2 = _run(W, P, dtype, False, calls, params)
    assert stb == W.WCNS_OK and st2 == W.WCNS_OK, (stb, st2)
    assert tb == t2 and nb == n2, (tb, t2, nb, n2)
    assert fbb == fb2, (fbb, fb2)
    diff = (ub != u2).sum().item()
    assert diff == 0, f"{diff} elements differ"


def test_banded_form_applies_only_to_large_2d_euler_grids(W):
    import torch
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        small = W.Solver(inputs.riemann2d(512, seed=0), "f32", stream=stream)
        with pytest.raises(W.WcnsError) as e:
            W.wcns_set_stage_form(small.ctx, True)
        assert e.value.status == W.WCNS_ERR_UNSUPPORTED
        W.wcns_set_stage_form(small.ctx, False)  # the two-launch form always applies
        small.close()
        line = W.Solver(inputs.sod(4096), "f64", stream=stream)
        with pytest.raises(W.WcnsError):
            W.wcns_set_stage_form(line.ctx, True)
        line.close()
        big = W.Solver(inputs.riemann2d(2048, seed=0, ny=700), "f32", stream=stream)
        W.wcns_set_stage_form(big.ctx, True)
        big.close()
        # only the default scheme configuration has banded kernels
        z = W.Solver(inputs.riemann2d(2048, seed=0, ny=700), "f32", stream=stream, weights="Z")
        with pytest.raises(W.WcnsError) as e:
            W.wcns_set_stage_form(z.ctx, True)
        assert e.value.status == W.WCNS_ERR_UNSUPPORTED
        z.close()
