import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA path through the C-ABI)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def oracle():
    from oracle import oracle as o
    o.build()
    return o


def pytest_terminal_summary(terminalreporter):
    """Every teacher-forced comparison of the session: rows judged, pass fraction
    and worst error / tolerance with the default magnitudes and with the narrower
    ones (sum |S I| for E, per-axis sums for dE/dc)."""
    P = sys.modules.get("tests._parity")
    log = getattr(P, "NARROW_LOG", None)
    if not log:
        return
    tr = terminalreporter
    tr.write_sep("-", "teacher-forced comparisons: default and narrower magnitudes")
    tr.write_line(f"{'rows':>8} {'pass':>9} {'worst':>7} {'narrow':>9} {'worst':>7}  test")
    for name, n, f, w, nf, nw in log:
        tr.write_line(f"{n:8d} {f:9.6f} {w:7.3f} {nf:9.6f} {nw:7.3f}  {name}")
    tr.write_line(f"lowest pass fraction with the narrower magnitudes: {min(x[4] for x in log):.6f} "
                  f"over {len(log)} comparisons")
