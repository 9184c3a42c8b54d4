import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def sdlib():
    """The CUDA library, built in-tree (fails loudly when it cannot be)."""
    import torch

    from paper_2503_11213_gb300 import build as B
    B.build()
    import paper_2503_11213_gb300 as sd
    sd.lib()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return sd
