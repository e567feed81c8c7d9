import os
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libsdfnn")


def _cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def sdf():
    """The CUDA library binding; builds libsdfnn if needed.  GPU tests only."""
    if not _cuda_available():
        pytest.fail("CUDA is not available: GPU tests need a GB300")
    from paper_2201_09147_gb300 import build, sdfnn
    build.build()
    sdfnn.lib()
    return sdfnn
