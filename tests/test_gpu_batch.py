"""Batched uneven 1D Euler problems (persistent kernels, captured graphs, autotuner)
against the oracle run on each problem alone."""
import numpy as np
import pytest

import oracle
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


def run_batch(W, sizes, offsets, u0, dtype, nsteps, tile=0, t_end=0.0, **params):
    import torch
    stream = torch.cuda.Stream()
    tdt = torch.float64 if dtype == "f64" else torch.float32
    code = W.WCNS_F64 if dtype == "f64" else W.WCNS_F32
    p = W.make_params(W.WCNS_EULER, code, **params)
    total = u0.shape[1]
    with torch.cuda.stream(stream):
        b = W.wcns_batch_init(offsets, sizes, total, 0.0, 1.0, W.WCNS_BC_TRANSMISSIVE, p, code, tile, stream)
        u = torch.as_tensor(u0).to(device="cuda", dtype=tdt).contiguous()
        W.wcns_batch_step(b, u, nsteps, t_end)
        out = u.double().cpu().numpy()
        times = W.wcns_batch_times(b, len(sizes))
        cfg = W.wcns_batch_config(b)
        st, nonph = W.wcns_batch_sync_status(b)
        W.wcns_batch_destroy(b)
    assert st == W.WCNS_OK, W.wcns_status_string(st)
    return out, times, cfg


def oracle_problem(u0, off, n, nsteps, t_end=0.0):
    P = inputs.Problem("p", 1, 3, int(n), 1, (0.0, 0.0), (1.0, 1.0), (1, 1),
                       u0[:, off:off + n][:, None, :].copy(), 1)
    u, t, taken, _ = oracle.step(P, nsteps=nsteps, t_end=t_end)
    return u[:, 0, :], t


def small_batch(seed=0, nprob=37):
    return inputs.batched_1d(nprob, seed=seed, nmin=10, nmax=1500)


@pytest.mark.parametrize("tile", [0, 123, 251, 507])
def test_batch_parity_f64(W, tile):
    sizes, offsets, u0 = small_batch()
    out, times, cfg = run_batch(W, sizes, offsets, u0, "f64", 5, tile=tile)
    assert cfg[0] in (123, 251, 507) and cfg[1] >= 1
    if tile == 0:
        assert cfg[2] >= 3  # the autotuner timed several candidates
    for k in range(len(sizes)):
        o, n = offsets[k], sizes[k]
        ref, tref = oracle_problem(u0, o, n, 5)
        got = out[:, o:o + n]
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < 1e-11, (k, n, err)
        assert abs(times[k] - tref) <= 1e-15 * tref


def test_batch_tiles_agree(W):
    """The tile only changes which block computes an interface, not the arithmetic (up to
    the compiler's FMA contraction choices in each instantiation)."""
    sizes, offsets, u0 = small_batch(seed=1)
    a, _, _ = run_batch(W, sizes, offsets, u0, "f64", 3, tile=123)
    b, _, _ = run_batch(W, sizes, offsets, u0, "f64", 3, tile=507)
    assert np.abs(a - b).max() / np.abs(a).max() < 1e-13


def test_batch_t_end_clipping(W):
    """Every problem lands exactly on t_end with its own step sequence; the state agrees to
    1e-11 or to within 10x the oracle's own change under a one-ulp input perturbation."""
    sizes, offsets, u0 = small_batch(seed=2, nprob=9)
    out, times, _ = run_batch(W, sizes, offsets, u0, "f64", 400, tile=251, t_end=0.01)
    assert np.all(times == 0.01)
    rng = np.random.default_rng(0)
    u0p = u0 * (1.0 + rng.choice([-1.0, 1.0], size=u0.shape) * 2.0 ** -52)
    for k in range(len(sizes)):
        o, n = offsets[k], sizes[k]
        ref, tref = oracle_problem(u0, o, n, 10 ** 6, t_end=0.01)
        refp, _ = oracle_problem(u0p, o, n, 10 ** 6, t_end=0.01)
        assert tref == 0.01
        sens = np.abs(refp - ref).max() / np.abs(ref).max()
        err = np.abs(out[:, o:o + n] - ref).max() / np.abs(ref).max()
        if err >= 1e-11:
            from parity import allow_sensitivity
            allow_sensitivity(err, sens, f"batch problem {k} to t=0.01")


def test_batch_f32_l1(W):
    sizes, offsets, u0 = small_batch(seed=3)
    out, _, _ = run_batch(W, sizes, offsets, u0, "f32", 20)
    for k in range(len(sizes)):
        o, n = offsets[k], sizes[k]
        ref, _ = oracle_problem(u0, o, n, 20)
        l1 = np.abs(out[:, o:o + n] - ref).mean(axis=1)
        assert np.all(l1 < 1e-3), (k, l1)


def test_batch_full_size_sampled(W):
    """4096 problems, N_k ~ U{64..8192} (about 16.9 M cells), FP32 and FP64 one step;
    20 sampled problems checked against the oracle."""
    sizes, offsets, u0 = inputs.batched_1d(4096, seed=0)
    assert 15e6 < sizes.sum() < 19e6
    rng = np.random.default_rng(0)
    pick = rng.choice(len(sizes), 20, replace=False)
    out64, _, _ = run_batch(W, sizes, offsets, u0, "f64", 1)
    out32, _, cfg = run_batch(W, sizes, offsets, u0, "f32", 1)
    for k in pick:
        o, n = offsets[k], sizes[k]
        ref, _ = oracle_problem(u0, o, n, 1)
        err = np.abs(out64[:, o:o + n] - ref).max() / np.abs(ref).max()
        assert err < 1e-11, (k, err)
        assert np.all(np.abs(out32[:, o:o + n] - ref).mean(axis=1) < 1e-3)

