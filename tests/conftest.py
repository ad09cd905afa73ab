import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: full-size parity case")


@pytest.fixture(scope="session")
def desc_lib():
    """libdesc.so, built in-tree if it is not there yet (nvcc cross-compiles
    without a GPU, so the host-only entry points are testable on CPU)."""
    from paper_2305_03448_gb300 import _build
    import paper_2305_03448_gb300 as D
    if not os.path.exists(D.LIB_PATH):
        _build.build()
    return D.lib()
