import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libsoc.so")
    config.addinivalue_line("markers", "slow: longer CPU statistical pins")


@pytest.fixture(scope="session")
def libsoc():
    """Build (if stale) and load libsoc.so; fails loudly when it cannot."""
    from paper_1812_06632_gb300 import build
    build.build()
    from paper_1812_06632_gb300 import soc
    return soc
