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
def gpu():
    """Build (if needed) and load libbrillouin.so; select cuda:0."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1012_3615_gb300 import abi, build

    build.build()
    abi.load()
    torch.cuda.set_device(0)
    return torch.device("cuda:0")


@pytest.fixture
def oracle_weights():
    """set the oracle's class weights for one test (restored afterwards)"""
    import oracle

    yield oracle.set_weights
    oracle.reset_weights()
