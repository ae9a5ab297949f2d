"""Approximate dispersion relation (Sec. 3.2, Eq. 22-28): the oracle's ADR is pinned to the
closed-form symbol of the linear fifth-order scheme where the FE map returns the ideal
weights; the GPU ADR (batched lines through wcns_rhs) matches the oracle's."""
import numpy as np
import pytest

from oracle import adr as oadr

D3 = (75 / 64, -25 / 384, 3 / 640)
C5 = np.array([3, -20, 90, 60, -5]) / 128.0


def linear_modified_wavenumber(alpha):
    """k(alpha) of the ideal-weight scheme: -symbol, with symbol = C(alpha) S(alpha)."""
    C = sum(C5[l + 2] * np.exp(1j * alpha * l) for l in range(-2, 3))
    S = sum(D3[m - 1] * (np.exp(1j * alpha * (m - 1)) - np.exp(-1j * alpha * m)) for m in (1, 2, 3))
    return C * S


def modes(n, count):
    ks = np.unique(np.linspace(1, n // 2 - 1, count).round().astype(int))
    return 2 * np.pi * ks / n


def test_oracle_adr_equals_linear_symbol_on_resolved_modes():
    n = 64
    alphas = 2 * np.pi * np.arange(1, 5) / n  # alpha <= 0.4: the weights sit on the ideal plateau
    kr, ki = oadr.adr(alphas, n)
    k = linear_modified_wavenumber(alphas)
    np.testing.assert_allclose(kr, k.real, atol=1e-12)
    np.testing.assert_allclose(ki, k.imag, atol=1e-12)


def test_oracle_adr_shape():
    """Low-wavenumber dispersion follows the exact k_i = alpha.  At xi = 1e6 the dissipation
    k_r is non-negative for every mode; at xi = 100 the map moves the ideal weights to
    (0.0666, 0.6081, 0.3253) (renormalised), a different linear scheme that is slightly
    anti-dissipative (k_r ~ -1e-5) on the lowest modes."""
    n = 64
    alphas = modes(n, 16)
    kr, ki = oadr.adr(alphas, n, xi=1e6)
    assert np.all(kr >= -1e-12) and abs(ki[0] - alphas[0]) < 1e-4
    kr, ki = oadr.adr(alphas, n, xi=100.0)
    assert np.all(kr[:3] > -1e-4) and np.all(kr[3:] > 0) and abs(ki[0] - alphas[0]) < 1e-4


@pytest.mark.gpu
@pytest.mark.parametrize("xi", [1e6, 100.0])
@pytest.mark.parametrize("weights", ["FE", "Z", "JS"])
def test_gpu_adr_matches_oracle(xi, weights):
    import torch
    from paper_2306_09760_gb300 import build as wbuild
    wbuild.build()
    from paper_2306_09760_gb300 import adr
    n = 64
    alphas = modes(n, 31)
    kr, ki = adr.gpu_adr(alphas, n, "f64", stream=torch.cuda.Stream(), xi=xi, weights=weights)
    okr, oki = oadr.adr(alphas, n, xi=xi, weights=weights)
    scale = np.max(np.abs(alphas))
    assert np.max(np.abs(kr - okr)) < 1e-11 * scale and np.max(np.abs(ki - oki)) < 1e-11 * scale
