"""Parity of the FE-WENO family (App. B) on the GPU with the oracle: the fifth-order
finite-difference WENO on Lax-Friedrichs split fluxes with the Z/FE weights and the
Table B.2 control rows, through the same sweep kernels (family = WENO)."""
import numpy as np
import pytest

import oracle
from paper_2306_09760_gb300 import inputs
from parity import check64

pytestmark = pytest.mark.gpu

WENO = dict(family="WENO")


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


def gpu_rhs(W, stream, P, dtype, **params):
    import torch
    with torch.cuda.stream(stream):
        S = W.Solver(P, dtype, stream=stream, **params)
        L = S.numpy(S.rhs()).astype(np.float64)
        st, nonph = S.status()
        S.close()
    assert st == W.WCNS_OK, W.wcns_status_string(st)
    return L, nonph


def gpu_steps(W, stream, P, dtype, nsteps, t_end=0.0, **params):
    import torch
    with torch.cuda.stream(stream):
        S = W.Solver(P, dtype, stream=stream, **params)
        S.step(0.0, nsteps, t_end)
        u = S.numpy().astype(np.float64)
        t, taken = S.time()
        st, _ = S.status()
        S.close()
    assert st == W.WCNS_OK, W.wcns_status_string(st)
    return u, t, taken


CASES = [
    ("advection_sine_200", lambda: inputs.advection_sine(200), {}),
    ("sod_4096", lambda: inputs.sod(4096), {}),
    ("shu_osher_1000_comp", lambda: inputs.shu_osher(1000), dict(characteristic=False)),
    ("riemann2d_300x130", lambda: inputs.riemann2d(300, seed=0, ny=130), {}),
    ("riemann2d_96x400_z", lambda: inputs.riemann2d(96, seed=1, ny=400), dict(weights="Z")),
    ("smooth2d_periodic_200x90", lambda: inputs.random_smooth_euler_2d(200, 90, seed=3), {}),
    ("piecewise1d_700_pfe", lambda: inputs.random_piecewise_euler_1d(700, seed=5), dict(weights="PFE", cv=1e-2)),
    ("piecewise1d_700_js", lambda: inputs.random_piecewise_euler_1d(700, seed=5), dict(weights="JS", eps=1e-6)),
]


@pytest.mark.parametrize("name,make,params", CASES, ids=[c[0] for c in CASES])
def test_weno_rhs_parity_f64(W, stream, name, make, params):
    P = make()
    prm = dict(WENO, **params)
    L, nonph = gpu_rhs(W, stream, P, "f64", **prm)
    Lr, _ = oracle.rhs(P, **prm)
    check64(L, Lr, lambda u0: oracle.rhs(P, u0, **prm)[0], P.u0, name, strict=True)
    assert nonph == 0


@pytest.mark.parametrize("name,make,params", CASES, ids=[c[0] for c in CASES])
def test_weno_rhs_parity_f32(W, stream, name, make, params):
    P = make()
    prm = dict(WENO, **params)
    L, _ = gpu_rhs(W, stream, P, "f32", **prm)
    Lr, _ = oracle.rhs(P, **prm)
    rel_l1 = np.abs(L - Lr).mean() / np.abs(Lr).mean()
    assert rel_l1 < 1e-4, rel_l1


def test_weno_sod_full_run(W, stream):
    """Sod to t = 0.2 (N = 1024): FP64 under the round-off criterion, FP32 in L1."""
    P = inputs.sod(1024)
    u, t, taken = gpu_steps(W, stream, P, "f64", 2000, 0.2, **WENO)
    ur, tr, takenr, _ = oracle.run_to(P, 0.2, **WENO)
    assert t == tr == 0.2 and taken == takenr
    check64(u, ur, lambda u0: oracle.run_to(P, 0.2, u=u0, **WENO)[0], P.u0, "weno sod")
    u32, _, _ = gpu_steps(W, stream, P, "f32", 2000, 0.2, **WENO)
    assert np.all(np.mean(np.abs(u32 - ur), axis=(1, 2)) < 1e-3)


def test_weno_2d_steps(W, stream):
    P = inputs.riemann2d(300, seed=0, ny=130)
    u, _, taken = gpu_steps(W, stream, P, "f64", 10, **WENO)
    ur, _, takenr, _ = oracle.step(P, nsteps=10, **WENO)
    assert taken == takenr == 10
    check64(u, ur, lambda u0: oracle.step(P, u0, nsteps=10, **WENO)[0], P.u0, "weno 2d")


def test_weno_periodic_conservation_gpu(W, stream):
    """The two-point difference telescopes: periodic sums are constant to round-off."""
    P = inputs.random_smooth_euler_2d(128, 96, seed=4)
    u, _, _ = gpu_steps(W, stream, P, "f64", 20, **WENO)
    s0, s1 = P.u0.sum(axis=(1, 2)), u.sum(axis=(1, 2))
    assert np.all(np.abs(s1 - s0) < 1e-12 * np.abs(P.u0).sum(axis=(1, 2)))


def test_weno_batch_parity(W):
    """The batched persistent path runs the WENO family too."""
    import torch
    sizes, offsets, u0 = inputs.batched_1d(23, seed=2, nmin=10, nmax=900)
    stream = torch.cuda.Stream()
    p = W.make_params(W.WCNS_EULER, W.WCNS_F64, **WENO)
    with torch.cuda.stream(stream):
        b = W.wcns_batch_init(offsets, sizes, u0.shape[1], 0.0, 1.0, W.WCNS_BC_TRANSMISSIVE, p, W.WCNS_F64, 0, stream)
        u = torch.as_tensor(u0).to(device="cuda").contiguous()
        W.wcns_batch_step(b, u, 4, 0.0)
        out = u.cpu().numpy()
        st, _ = W.wcns_batch_sync_status(b)
        W.wcns_batch_destroy(b)
    assert st == W.WCNS_OK
    for k in range(len(sizes)):
        o, n = offsets[k], sizes[k]
        P = inputs.Problem("p", 1, 3, int(n), 1, (0.0, 0.0), (1.0, 1.0), (1, 1), u0[:, o:o + n][:, None, :].copy(), 1)
        ref = oracle.step(P, nsteps=4, **WENO)[0][:, 0, :]
        err = np.abs(out[:, o:o + n] - ref).max() / np.abs(ref).max()
        assert err < 1e-11, (k, n, err)


def test_weno_adjoint_is_unsupported(W):
    import torch
    P = inputs.vortex(32, seed=1)
    S = W.Solver(P, "f64", flux="LLF_FROZEN", alpha=(3.0, 3.0), **WENO)
    lam = torch.zeros_like(S.u)
    with pytest.raises(W.WcnsError) as e:
        W.wcns_adjoint_step(S.ctx, S.u, 1e-3, lam, lam)
    assert e.value.status == W.WCNS_ERR_UNSUPPORTED
    S.close()
