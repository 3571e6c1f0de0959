import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")


import pytest


@pytest.fixture(scope="session")
def gpu():
    """(binding module, torch) with the CUDA library built and a GPU present."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_2601_10981_gb300 import build as _build
    import os
    if not os.path.exists(_build.lib_path()):
        _build.build()
    from paper_2601_10981_gb300 import binding
    binding.lib()
    return binding, torch
