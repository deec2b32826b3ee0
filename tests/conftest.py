"""Shared pytest setup: the `gpu` marker and import paths."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size workload, minutes")


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def gpu():
    """The product library, loaded on a GPU machine.  Fails loudly when the GPU is
    there but the CUDA extension is not."""
    if not cuda_available():
        pytest.skip("no CUDA device")
    import paper_1209_6007_gb300 as bcs
    bcs.load()  # raises if libbcshatter.so is missing
    return bcs
