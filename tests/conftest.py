import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


def _cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def gpu():
    """The CUDA binding, built for sm_103a; the test fails loudly without it."""
    if not _cuda_ok():
        pytest.fail("GPU test selected but no CUDA device is visible")
    from paper_2505_21728_gb300 import build as hb
    hb.build()
    from paper_2505_21728_gb300 import hygt
    return hygt
