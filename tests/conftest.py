import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU check")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


def pytest_runtest_teardown(item, nextitem):
    """With DQ_PARITY_LOG set, append every result's max-abs and max-rel error
    against the oracle (one JSON line per checked result) to that file."""
    path = os.environ.get("DQ_PARITY_LOG")
    mod = sys.modules.get("tests.gpu_helpers")
    if path and mod is not None and mod.RECORDS:
        mod.write_records(path)
