"""Writes the algorithmic flop count per cell of one RHS evaluation of the benchmark's
2D Euler workload to profiles/algorithmic_flops.json.

The count is the oracle's exact operation count (one flop per +, -, *, /, sqrt, tanh)
of its plain restatement of the method (Eq. 3-6, 9-15, 20-21; Roe-averaged
characteristic projection, HLLC) on a 64 x 64 sample of the same four-quadrant data,
divided by the number of cells.  The benchmark's roofline line reads the stored value,
so the timed program runs no oracle code.

Usage: python -m oracle.write_flop_counts
"""
from __future__ import annotations

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "profiles", "algorithmic_flops.json")


def main() -> None:
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle
    from paper_2306_09760_gb300 import inputs
    oracle.build()
    n = 64
    P = inputs.riemann2d(n, seed=0)
    per_cell = oracle.count_rhs_flops(P) / (P.nx * P.ny)
    d = {"_doc": "Exact operation count of one RHS evaluation per cell (both sweep directions), "
                 "from the oracle on a 64 x 64 sample of the 2D four-quadrant Riemann workload (seed 0, "
                 "WCNS-FE xi = 1e6, HLLC, characteristic). Written by oracle/write_flop_counts.py.",
         "euler2d_riemann_rhs_flops_per_cell": per_cell}
    with open(OUT, "w") as f:
        json.dump(d, f, indent=1)
        f.write("\n")
    print(OUT, per_cell)


if __name__ == "__main__":
    main()
