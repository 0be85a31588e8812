import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def ora():
    import oracle
    oracle.lib()
    return oracle


@pytest.fixture(autouse=True)
def _bounds_check_record(request):
    """With AIRGA_LIB=checked (the bounds-checked library) every GPU test
    ends by reading the library's record of out-of-range indices: a test
    whose kernels addressed outside a buffer errors in teardown."""
    yield
    if os.environ.get("AIRGA_LIB") != "checked" or request.node.get_closest_marker("gpu") is None:
        return
    A = sys.modules.get("paper_1606_01216_gb300.airga")
    if A is None or A._lib is None:
        return
    v, site, idx = A.debug_checked()
    assert v == 0, "%d out-of-range index(es); one at check site %d, index %d" % (v, site, idx)
