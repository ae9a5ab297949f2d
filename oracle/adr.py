"""ADR (Sec. 3.2, Eq. 22-28) of the oracle's spatial operator -- TEST INFRASTRUCTURE ONLY.

Each Fourier mode cos(alpha x) on a periodic grid of n points (h = 1, c = 1) goes through
the oracle's RHS on its own; the modified wavenumber k = k_r + i k_i (Eq. 28) is the
Fourier coefficient of the numerical derivative u_x h = -L at alpha divided by that of
the mode.  The exact derivative gives (k_r, k_i) = (0, alpha) (Eq. 27); k_i is the
dispersion and k_r >= 0 the dissipation (the mode decays like exp(-c k_r t / h)).
"""
from __future__ import annotations

import numpy as np

from . import rhs
from paper_2306_09760_gb300 import inputs


def adr(alphas, n=64, **params):
    x = np.arange(n)
    kr = np.zeros(len(alphas))
    ki = np.zeros(len(alphas))
    for j, a in enumerate(alphas):
        u0 = np.cos(a * x)[None, None, :].copy()
        P = inputs.Problem("adr", 1, 1, n, 1, (0.0, 0.0), (float(n), 1.0), (0, 0), u0, 0, adv_speed=(1.0, 0.0))
        L, _ = rhs(P, **params)
        d = -L[0, 0]
        # Fourier coefficient of d at alpha over that of cos(alpha x) (which is n/2)
        k = np.sum(d * np.exp(-1j * a * x)) / (n / 2.0)
        kr[j], ki[j] = k.real, k.imag
    return kr, ki
