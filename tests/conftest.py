import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(autouse=True)
def _reset_oracle_hooks():
    """Every test starts and ends with a faithful oracle."""
    yield
    if "oracle.oracle" in sys.modules:
        import oracle
        oracle.set_mutation(0)
        oracle.set_paranoid(False)
