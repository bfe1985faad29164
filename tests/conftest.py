import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# the oracle mutation test points this at a copy of oracle/ with one planted
# mistake, so that the pins run against the mutant
_MUTANT = os.environ.get("RELSIM_ORACLE_MUTANT_DIR")
if _MUTANT:
    sys.path.insert(0, _MUTANT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.load()
    return oracle
