import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def error_report():
    """Error of the GPU path against the FP64 oracle, per workload, collected
    by the parity tests; written as JSON to $MGS_ERROR_REPORT when set."""
    import json
    rows = {}
    yield rows
    path = os.environ.get("MGS_ERROR_REPORT")
    if path and rows:
        with open(path, "w") as f:
            json.dump(rows, f, indent=1, sort_keys=True)
