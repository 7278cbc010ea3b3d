import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# The property-based host tests need hypothesis, which not every machine has;
# where it is missing the module is left out of collection (it holds no GPU
# test) instead of showing up as a skipped module.
try:
    import hypothesis  # noqa: F401
except ImportError:
    collect_ignore = ["test_properties.py"]


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a); run with -m gpu")
    config.addinivalue_line("markers", "slow: large host-side case")


@pytest.fixture(scope="session")
def golden_dir():
    return os.path.join(ROOT, "tests", "golden")
