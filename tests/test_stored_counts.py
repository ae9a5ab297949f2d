"""The algorithmic flop count that the benchmark's roofline line reads from
profiles/algorithmic_flops.json equals the oracle's exact operation count now."""
import json
import os

import oracle
from paper_2306_09760_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_stored_flop_count_matches_oracle():
    with open(os.path.join(ROOT, "profiles", "algorithmic_flops.json")) as f:
        stored = json.load(f)["euler2d_riemann_rhs_flops_per_cell"]
    P = inputs.riemann2d(64, seed=0)
    assert oracle.count_rhs_flops(P) / (P.nx * P.ny) == stored
