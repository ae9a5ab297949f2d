"""Host check of the FE-map tables the library gives its kernels (no GPU).

`tests/tables_check.cu` builds the library's `fill_family_tables` as a host program and
prints, for the WCNS family (Table 2) and the FE-WENO family (Table B.2) at kappa = 1/2,
the ideal weights, the null points of Eq. 20 and the control values of its plateaus.
They are compared with what the paper prints in Table 1 and Table B.1 (the golden files):
the ideal weights are the Case0 rows; each weight's plateaus take the control values of
its control points in ascending order; and the null points kappa (psi_j + psi_{j-1}) are
the midpoints of consecutive entries of 0, the control points and 1 (Eq. 20 is the
identity beyond the last control point, so the map of every weight ends at 1).
"""
from fractions import Fraction
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")
FILES = {0: "table1_control_values.txt", 1: "tableB1_control_values.txt"}


def _golden(family):
    rows = []
    with open(os.path.join(GOLDEN, FILES[family])) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                case, i, orig, mapped = line.split()
                rows.append((case, int(i), Fraction(orig), Fraction(mapped)))
    return rows


def _expected(family):
    rows = _golden(family)
    ideal = [next(o for c, i, o, m in rows if c == "Case0" and i == k) for k in range(3)]
    nulls, ctrls = {}, {}
    for k in range(3):
        pts = sorted({(o, m) for c, i, o, m in rows if i == k and o < 1})
        psi = [Fraction(0)] + [o for o, _ in pts] + [Fraction(1)]
        nulls[k] = [(psi[j] + psi[j - 1]) / 2 for j in range(1, len(psi))]
        ctrls[k] = [m for _, m in pts]
    return ideal, nulls, ctrls


@pytest.fixture(scope="module")
def tables():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "tables_check")
        r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-x", "cu", "-o", exe,
                            os.path.join(HERE, "tables_check.cu")], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    t = {}
    for line in out.stdout.split("\n"):
        if line.strip():
            f = line.split()
            t[(int(f[0]), f[1])] = [float(x) for x in f[2:]]
    return t


@pytest.mark.parametrize("family", [0, 1])
def test_library_tables_match_the_printed_control_values(tables, family):
    ideal, nulls, ctrls = _expected(family)
    assert tables[(family, "ideal")] == [float(x) for x in ideal]
    for k in range(3):
        got = tables[(family, f"null{k}")]
        assert len(got) == len(nulls[k]), (k, got)
        for g, w in zip(got, nulls[k]):
            assert abs(g - float(w)) <= 2e-16, (family, k, got, nulls[k])
        assert tables[(family, f"ctrl{k}")] == [float(x) for x in ctrls[k]], (family, k)
        # the first plateau is the ideal weight's own
        assert ctrls[k][0] == ideal[k]
