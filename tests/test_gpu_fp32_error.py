"""FP32 bulk arithmetic against the FP64 oracle, per configuration of the workload.

For each configuration the FP32 GPU path runs the configuration's own run (length,
step rule, scheme) and its final state is compared with the oracle's: relative L1 per
conserved variable, mean |u32 - u64| / mean |u64|, at most 1e-5 on smooth data and
1e-3 on shocked data (the relative form keeps the bound meaningful across variables of
different size: density ~1, energy ~2.5-10).  Smooth runs also get a per-element bound
(no captured discontinuity can move a cell there).  The oracle runs in spawned worker
processes while the GPU works.
"""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np
import pytest

from paper_2306_09760_gb300 import inputs
from parity import L1_SHOCKED, L1_SMOOTH, rel_l1

pytestmark = pytest.mark.gpu

# adjoint workload parameters (frozen LLF at the initial maximum wave speed, constant dt)
_C5 = inputs.vortex(512, seed=0)
_c = np.sqrt(1.4 * _C5.extra["p"] / _C5.extra["rho0"])
_AMAX = float(max((np.abs(_C5.extra["u"]) + _c).max(), (np.abs(_C5.extra["v"]) + _c).max()))
C5_PARAMS = dict(flux="LLF_FROZEN", alpha=(_AMAX, _AMAX), xi=100.0, zp=2, characteristic=True, eps=1e-4)
C5_DT = 0.5 * _C5.h[0] / _AMAX

# name, steps, t_end, fixed dt (<= 0: CFL), scheme parameters, smooth?
CONFIGS = [
    ("C1_advection_200", 500, 2.0, 0.0, {}, True),
    ("C2a_sod_4096", 10 ** 6, 0.2, 0.0, {}, False),
    ("C2b_shu_osher_4096", 10 ** 6, 1.8, 0.0, {}, False),
    ("C3_riemann2d_256", 100, 0.0, 0.0, {}, False),
    ("C5_vortex_512", 200, 0.0, C5_DT, C5_PARAMS, True),
    ("titarev_toro_2001", 400, 0.0, 0.0, {}, False),
]


@pytest.fixture(scope="module")
def oracle_futures():
    """Starts every oracle run in a spawned worker pool before the first GPU call."""
    import oracle
    oracle.build()
    import oracle_runs
    cores = os.cpu_count() or 4
    ex = cf.ProcessPoolExecutor(max_workers=3, mp_context=mp.get_context("spawn"))
    futs = {name: ex.submit(oracle_runs.run, name, n, t_end, dt, params, max(1, cores // 2))
            for name, n, t_end, dt, params, _ in CONFIGS}
    yield futs
    ex.shutdown(wait=True, cancel_futures=True)


@pytest.fixture(scope="module")
def W(oracle_futures):
    import torch
    assert torch.cuda.is_available()
    from paper_2306_09760_gb300 import build as wbuild
    wbuild.build()
    from paper_2306_09760_gb300 import wcns
    return wcns


@pytest.mark.parametrize("name,nsteps,t_end,dt,params,smooth", CONFIGS, ids=[c[0] for c in CONFIGS])
def test_fp32_error_per_config(W, oracle_futures, name, nsteps, t_end, dt, params, smooth):
    import oracle_runs
    import torch
    P = oracle_runs._problem(name)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        S = W.Solver(P, "f32", stream=stream, **params)
        S.step(dt, nsteps, t_end)
        u32 = S.numpy()
        t32, taken32 = S.time()
        st, _ = S.status()
        S.close()
    assert st == W.WCNS_OK
    ur, tr, takenr = oracle_futures[name].result()
    if t_end > 0:
        assert abs(t32 - t_end) < 1e-12 and tr == t_end
    else:
        assert taken32 == takenr == nsteps
    l1 = rel_l1(u32, ur)
    emax = np.abs(u32 - ur).max(axis=tuple(range(1, ur.ndim))) / np.abs(ur).max(axis=tuple(range(1, ur.ndim)))
    print(f"\nFP32 vs oracle {name}: relative L1 per variable {[f'{x:.2e}' for x in l1]}, "
          f"relative max {[f'{x:.2e}' for x in emax]}, steps {taken32} / {takenr}")
    bound = L1_SMOOTH if smooth else L1_SHOCKED
    assert np.all(l1 < bound), (name, l1, bound)
    if smooth:
        assert np.all(emax < 1e-4), (name, emax)
