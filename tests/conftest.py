import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(autouse=True)
def _debug_build_flags(request):
    """Under the bounds-checked library (FLD_LIBRARY naming libfld_gb300_debug.so) every GPU
    test must leave no bounds flag raised."""
    yield
    lib = os.environ.get("FLD_LIBRARY", "")
    if lib.endswith("_debug.so") and request.node.get_closest_marker("gpu"):
        from paper_2503_02764_gb300 import fld
        assert fld.fld_debug_flags() == 0, "a kernel indexed outside its array"
