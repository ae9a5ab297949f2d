"""Shared FP64 parity criterion of the GPU tests.

The GPU and the oracle round differently (FMA contraction, factored eigenvector
products, CUDA's tanh/sqrt), so they agree to the last bits only where the scheme is
well conditioned.  Two places are not: (1) long shocked runs, where the nonlinear
weights amplify round-off step after step; (2) stretches of exactly constant data
next to a jump, where IS ~ 1e-33 from round-off dwarfs eps = 1e-40 and so decides the
Z weights.  The criterion is therefore: relative max error below 1e-11, or below ten
times the oracle's own change when every input value moves by one ulp (the
round-off amplification any correct implementation must be allowed).  The
sensitivity is computed only when the strict bound is missed.
"""
import numpy as np

TOL64 = 1e-11


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def perturb_ulp(u0, seed=0):
    rng = np.random.default_rng(seed)
    return u0 * (1.0 + rng.choice([-1.0, 1.0], size=u0.shape) * 2.0 ** -52)


def check64(got, ref, run_oracle, u0, what=""):
    """run_oracle(u0) -> oracle result for input u0 (the unperturbed one gives ref)."""
    err = rel_max(got, ref)
    if err < TOL64:
        return err
    sens = rel_max(run_oracle(perturb_ulp(u0)), ref)
    assert err < 10.0 * sens, f"{what}: GPU vs oracle {err:.3e}, oracle 1-ulp sensitivity {sens:.3e}"
    return err
