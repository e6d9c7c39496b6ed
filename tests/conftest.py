import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture
def repo_tmp():
    """A scratch directory inside the repository (git-ignored), removed after the test."""
    import shutil
    import tempfile
    base = os.path.join(ROOT, ".pytest_tmp")
    os.makedirs(base, exist_ok=True)
    path = tempfile.mkdtemp(dir=base)
    yield path
    shutil.rmtree(path, ignore_errors=True)
