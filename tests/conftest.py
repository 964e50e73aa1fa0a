import os
import sys

import pytest

# The oracle's OpenMP threads sleep between its parallel loops instead of spinning, so that the
# numpy work a test does between oracle steps does not compete with them for the cores (set
# before any OpenMP runtime is loaded; an explicit setting in the environment wins).
os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA path through the C ABI)")
    config.addinivalue_line("markers", "slow: longer CPU oracle runs")


@pytest.fixture(scope="session")
def cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1705_03141_gb300 as pkg

    pkg.build_library()
    pkg.library()
    return torch.device("cuda", 0)
