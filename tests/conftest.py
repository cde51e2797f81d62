import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle


@pytest.fixture(scope="session", autouse=True)
def bounds_check_session():
    """With ALB_BOUNDS_CHECK=1 the GPU tests run on the bounds-checked build
    of the library; after the session no instrumented access may have left
    its region."""
    yield
    if os.environ.get("ALB_BOUNDS_CHECK", "") != "1":
        return
    from paper_1809_06839_gb300 import alb
    if alb._lib is None:
        return
    checked, count, line = alb.alb_bounds_violations()
    assert checked, "ALB_BOUNDS_CHECK=1 but the loaded library is not the checked build"
    assert count == 0, f"{count} bounds violations, first at source line {line}"
