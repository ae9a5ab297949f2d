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


def test_kernel_digest_follows_code_not_comments():
    """The digest that ties the stored DRAM counters to the captured kernels changes with
    the code and not with comments or white space."""
    import bench
    src = {n: open(os.path.join(ROOT, "paper_2306_09760_gb300", "csrc", n), "rb").read()
           for n in bench.SWEEP_SOURCES}
    base = bench.kernel_source_digest(src.__getitem__)
    name = bench.SWEEP_SOURCES[2]
    edited = dict(src)
    edited[name] = b"// a new comment\n/* and a block\n comment */\n" + src[name].replace(b";\n", b";  \n\n", 3)
    assert bench.kernel_source_digest(edited.__getitem__) == base
    changed = dict(src)
    changed[name] = src[name].replace(b"kYPer = 5", b"kYPer = 6", 1)
    assert changed[name] != src[name]
    assert bench.kernel_source_digest(changed.__getitem__) != base
    lit = dict(src)
    lit[name] = src[name].replace(b'"fence.proxy.async.shared::cta;"', b'"fence.proxy.async.shared::cta; "', 1)
    assert lit[name] != src[name]
    assert bench.kernel_source_digest(lit.__getitem__) != base  # string literals are code
