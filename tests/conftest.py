import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test")


import pytest


@pytest.fixture(autouse=True)
def _range_checked_run(request):
    """Under MG5_BOUNDS=1 (the range-checked library) every GPU test ends by reading the
    library's record of out-of-range accesses: any entry fails the test."""
    yield
    if os.environ.get("MG5_BOUNDS", "0") != "1" or request.node.get_closest_marker("gpu") is None:
        return
    import torch
    import paper_1511_08200_gb300 as mg
    torch.cuda.synchronize()
    msg = mg.bounds_check()
    assert msg is None, "out-of-range access: %s" % msg
