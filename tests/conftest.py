import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built C-ABI library")
    config.addinivalue_line("markers", "slow: long-running oracle comparison")


def read_golden(name):
    """Rows of a golden fixture file, comments stripped."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line)
    return rows


@pytest.fixture(scope="session")
def lib():
    """The C-ABI library, built in-tree on first use."""
    from paper_2412_08229_gb300 import _abi
    return _abi.load(build_if_missing=True)
