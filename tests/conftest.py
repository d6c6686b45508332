import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


import pytest


@pytest.fixture(autouse=True)
def _one_step_path_unless_selected(request, monkeypatch):
    """GPU tests run the one-step kernels (and their variants) unless the
    environment or the test itself selects the two-step path; the two-step
    path has its own tests (test_gpu_tb.py), which set FDTD_TB."""
    if request.node.get_closest_marker("gpu") is not None and "FDTD_TB" not in os.environ:
        monkeypatch.setenv("FDTD_TB", "0")
