import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


_MEASUREMENTS = []


@pytest.fixture(scope="session")
def measurements():
    """Tests append one-line results (times, speed-ups) here; they are printed in the
    terminal summary, so a quiet run (-q) still shows them."""
    return _MEASUREMENTS


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    if _MEASUREMENTS:
        terminalreporter.section("measurements")
        for line in _MEASUREMENTS:
            terminalreporter.write_line(line)
