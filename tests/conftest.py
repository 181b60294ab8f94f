import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (sm_103a) and the built libtomo")


@pytest.fixture(scope="session")
def golden_dir():
    return os.path.join(ROOT, "tests", "golden")


def pytest_terminal_summary(terminalreporter):
    """Share of the compared elements that met the parity bound only through
    its absolute term (gpu_util.FLOOR_SHARES), per check."""
    try:
        from tests.gpu_util import FLOOR_SHARES
    except ImportError:
        return
    if not FLOOR_SHARES:
        return
    tr = terminalreporter
    tr.write_sep("-", "parity: elements inside the bound only by its absolute term")
    worst = max(FLOOR_SHARES, key=lambda r: r[1] / max(r[2], 1))
    total = sum(r[1] for r in FLOOR_SHARES), sum(r[2] for r in FLOOR_SHARES)
    for what, n_floor, n in FLOOR_SHARES:
        if n_floor:
            tr.write_line("%-48s %9d of %11d (%.2e)" % (what[:48], n_floor, n,
                                                        n_floor / max(n, 1)))
    tr.write_line("all checks: %d of %d (%.2e); worst %s at %.2e"
                  % (total[0], total[1], total[0] / max(total[1], 1),
                     worst[0], worst[1] / max(worst[2], 1)))
