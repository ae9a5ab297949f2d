"""Host check of the FE ideal-plateau margins (no GPU).

The kernels skip Eq. 20 where every base weight lies within a margin of its ideal weight
d_k (or, before the Z weights are normalised, where every ratio of Eq. 14 is below a
bound), returning the ideal weights directly.  `tests/margins_check.cu` builds the
library's own host derivation of those margins (`scheme_as` / `ideal_margins`) as a
host program; here they are checked against the oracle's evaluation of Eq. 20:

* inside the margin the oracle's map returns the ideal weight (to the last bit in FP64,
  to the tanh saturation of single precision in FP32);
* Z weights whose ratios are all below the ratio bound stay inside the margins;
* the margins are nearly tight: just past them the map has left the plateau;
* the test is off exactly where the map does not return the ideal weights (small xi,
  kappa = 0.3 of Sec. 3.2) and for PFE, whose App. A box keeps the Z weights.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
IDEAL = {0: (1 / 16, 10 / 16, 5 / 16), 1: (1 / 10, 6 / 10, 3 / 10)}  # Table 2 / Table B.2


def _map(family):
    return oracle.fe_map if family == 0 else oracle.fe_map_weno


@pytest.fixture(scope="module")
def rows():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "margins_check")
        r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-x", "cu", "-o", exe,
                            os.path.join(HERE, "margins_check.cu")], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    parsed = []
    for line in out.stdout.split("\n"):
        if line.strip():
            f = line.split()
            parsed.append(dict(bytes=int(f[0]), family=int(f[1]), xi=float(f[2]), kappa=float(f[3]),
                               weights=int(f[4]), m=[float(x) for x in f[5:8]], ratio=float(f[8]),
                               sat=float(f[9])))
    assert len(parsed) == 2 * 6 * 2 * 2 * 2
    return parsed


def _tol(row):
    # FP64: the saturated map is exact; FP32: single-precision tanh is exactly 1 from 9.1 on,
    # where the double-precision map still differs by at most e^-18.2 of a term's amplitude
    return 1e-15 if row["bytes"] == 8 else 3e-8


def _on(row):
    return row["weights"] == 2 and all(m > 0 for m in row["m"]) and row["ratio"] > 0


def test_margins_on_where_expected(rows):
    """The test is on for FE weights at kappa = 1/2 once xi is large enough for a saturated
    plateau around every d_k, and off for PFE and for kappa = 0.3."""
    for r in rows:
        if r["weights"] == 3 or r["kappa"] != 0.5:
            assert r["m"] == [0.0, 0.0, 0.0] and r["ratio"] == 0.0, r
        elif r["xi"] >= 1e4:
            assert _on(r), r
        if r["bytes"] == 4 and r["xi"] < 1e4:
            assert not _on(r), r  # single precision evaluates the small-xi map in exponential form


def test_map_returns_ideal_weights_inside_the_margins(rows):
    for r in rows:
        if not _on(r):
            continue
        g = _map(r["family"])
        for k, d in enumerate(IDEAL[r["family"]]):
            m = r["m"][k]
            for w in (d - m, d - 0.5 * m, d, d + 0.5 * m, d + m):
                assert abs(g(k, w, xi=r["xi"], kappa=r["kappa"]) - d) <= _tol(r), (r, k, w)


def test_ratio_bound_keeps_z_weights_inside_the_margins(rows):
    """Eq. 14: w_k = d_k (1 + r_k) / (1 + sum_l d_l r_l); with every r_l in [0, rho) each w_k
    is within d_k rho of d_k, inside the margin, so the map returns d_k there too."""
    rng = np.random.default_rng(5)
    for r in rows:
        if not _on(r):
            continue
        d = np.array(IDEAL[r["family"]])
        rho = r["ratio"]
        corners = [np.array(c, dtype=float) * rho * (1 - 1e-12)
                   for c in ((1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (0, 1, 1), (1, 0, 1), (1, 1, 1))]
        for rr in corners + [rng.uniform(0, rho, 3) for _ in range(50)]:
            w = d * (1 + rr) / (1 + (d * rr).sum())
            assert np.all(np.abs(w - d) <= np.array(r["m"])), (r, rr, w)
            g = _map(r["family"])
            for k in range(3):
                assert abs(g(k, w[k], xi=r["xi"], kappa=r["kappa"]) - d[k]) <= _tol(r)


def test_margins_are_nearly_tight(rows):
    """A little past the margin (two saturation distances and the rounding allowance) the
    map has crossed a null point on at least one side of d_k, for every k."""
    for r in rows:
        if not _on(r):
            continue
        g = _map(r["family"])
        for k, d in enumerate(IDEAL[r["family"]]):
            past = r["m"][k] + 2.2 * r["sat"] + 3e-6
            dev = max(abs(g(k, d - past, xi=r["xi"], kappa=r["kappa"]) - d),
                      abs(g(k, d + past, xi=r["xi"], kappa=r["kappa"]) - d))
            assert dev > 1e-3, (r, k, dev)


def test_off_where_the_map_leaves_the_ideal_weights(rows):
    """Where the library turns the test off for FE weights in double precision (xi of 100 or
    1000, kappa = 0.3), the oracle's map does not return every ideal weight exactly, so the
    shortcut would change results there."""
    for r in rows:
        if r["weights"] != 2 or r["bytes"] != 8 or _on(r):
            continue
        g = _map(r["family"])
        dev = max(abs(g(k, d, xi=r["xi"], kappa=r["kappa"]) - d) for k, d in enumerate(IDEAL[r["family"]]))
        assert dev > 1e-16, r
