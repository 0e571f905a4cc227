import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(autouse=True)
def _bounds_checked_build_stays_clean():
    """Under FRP_BOUNDS_CHECK=1 (the bounds-checked library), no field of a
    test may end with a fired partner-index check (FR_EBOUNDS)."""
    yield
    if os.environ.get("FRP_BOUNDS_CHECK") == "1":
        import gc
        gc.collect()
        from paper_2006_10967_gb300 import _capi
        assert not _capi.BOUNDS_FIRED, f"partner index check fired in {len(_capi.BOUNDS_FIRED)} field(s)"
