import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

_REPORT = []


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def report_lines():
    """Lines a test wants shown in the terminal summary (measured error reports)."""
    return _REPORT


def pytest_terminal_summary(terminalreporter):
    if _REPORT:
        terminalreporter.section("measured reports")
        for line in _REPORT:
            terminalreporter.write_line(line)
