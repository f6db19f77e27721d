import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU check")


@pytest.fixture(scope="session")
def cuda_lib():
    """The CUDA library's binding, built in-tree; skips cleanly without a GPU."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1106_1900_gb300 as bh

    bh.load()
    return bh
