import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels)")
    config.addinivalue_line("markers", "slow: longer test")


@pytest.fixture(scope="session", autouse=True)
def _native_builds():
    """Compile the oracle, the input generators and the C-ABI library (release and bounds-checked
    debug builds) if they are stale."""
    import oracle
    from paper_2603_28796_b300 import build

    oracle.build()
    build.build_synth()
    build.build_library()
    build.build_library(debug=True)
    yield
