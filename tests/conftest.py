import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Lists the FP64 checks that passed only through the multi-step round-off allowance."""
    import parity
    if parity.FALLBACKS:
        terminalreporter.section("FP64 parity: checks that used the one-ulp sensitivity allowance")
        for what, err, sens in parity.FALLBACKS:
            terminalreporter.write_line(f"{what}: GPU vs oracle {err:.3e}, oracle 1-ulp sensitivity {sens:.3e} "
                                        f"(ratio {err / sens:.2f})")
