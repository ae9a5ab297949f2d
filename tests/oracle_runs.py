"""Oracle runs of the FP32 error tests, executed in worker processes.

The workers are started with the "spawn" method, so they share no CUDA state with the
test process (the GPU runs alongside them).  Each job returns the oracle's final state.
"""
from __future__ import annotations


def _problem(name):
    from paper_2306_09760_gb300 import inputs
    if name == "C1_advection_200":
        return inputs.advection_sine(200)
    if name == "C2a_sod_4096":
        return inputs.sod(4096)
    if name == "C2b_shu_osher_4096":
        return inputs.shu_osher(4096)
    if name == "C3_riemann2d_256":
        return inputs.riemann2d(256, seed=0)
    if name == "C5_vortex_512":
        return inputs.vortex(512, seed=0)
    if name == "titarev_toro_2001":
        return inputs.titarev_toro(2001)
    raise KeyError(name)


def run(name, nsteps, t_end, dt, params, threads):
    """Oracle state after nsteps TVD-RK3 steps (CFL steps if dt <= 0, clipped at t_end)."""
    import oracle
    oracle.set_threads(threads)
    P = _problem(name)
    u, t, taken, _ = oracle.step(P, dt=dt, nsteps=nsteps, t_end=t_end, **params)
    return u, t, taken
