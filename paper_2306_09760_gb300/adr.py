"""Approximate dispersion relation (ADR) of the nonlinear scheme (Sec. 3.2, Eq. 22-28).

For u_t + c u_x = 0 and an initial Fourier mode of wavenumber alpha = omega * dx, the
scheme's spatial operator gives a numerical derivative whose Fourier coefficient at alpha,
relative to that of the mode, is the modified wavenumber k = k_r + i k_i (Eq. 28); the
exact derivative gives k_r = 0, k_i = alpha (Eq. 27).  Because the weights are nonlinear,
each mode is evaluated on its own: line j of a batch holds cos(alpha_j x) on a periodic
grid of n points, and all lines go through one wcns_rhs call of the library (ndim 1,
ny = number of modes):  k_j = (2 / n) sum_x (-L h / c) e^{-i alpha_j x}.
"""
from __future__ import annotations

import numpy as np

from . import inputs, wcns


def mode_lines(alphas, n):
    """[1, nmodes, n] array of cos(alpha_j * x), x = 0..n-1 (periodic only when
    alpha_j * n is a multiple of 2 pi, which `modes` guarantees)."""
    x = np.arange(n)
    return np.cos(np.outer(alphas, x))[None, :, :]


def modes(n, count):
    """`count` wavenumbers 2 pi k / n spread over (0, pi]."""
    ks = np.unique(np.linspace(1, n // 2, count).round().astype(int))
    return 2.0 * np.pi * ks / n


def modified_wavenumber(L, alphas, n, c=1.0, h=1.0):
    """(k_r, k_i) per mode from RHS lines L [nmodes, n]."""
    x = np.arange(n)
    D = -L * h / c  # numerical u_x h
    k = (2.0 / n) * np.sum(D * np.exp(-1j * np.outer(alphas, x)), axis=1)
    return k.real, k.imag


def gpu_adr(alphas, n=64, dtype="f64", stream=None, **params):
    """Modified wavenumbers of the FE scheme (or any weights) from the CUDA path."""
    u0 = mode_lines(alphas, n)
    P = inputs.Problem("adr", 1, 1, n, len(alphas), (0.0, 0.0), (float(n), 1.0), (0, 0), u0, 0,
                       adv_speed=(1.0, 0.0))
    S = wcns.Solver(P, dtype, stream=stream, **params)
    L = S.numpy(S.rhs())[0]
    S.close()
    kr, ki = modified_wavenumber(L, alphas, n)
    return kr, ki
