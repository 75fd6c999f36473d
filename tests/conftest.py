import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _build_libraries():
    """Compile the CUDA library and the C oracle if their sources changed."""
    import oracle
    oracle.build()
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "cetra_build", os.path.join(ROOT, "paper_2503_20875_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)  # the build script alone: the package needs the library it builds
    b.build()


def pytest_configure(config):
    _build_libraries()
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if gpu_available():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)
