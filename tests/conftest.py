import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def built_lib():
    """Builds libtp.so in-tree (nvcc cross-compiles without a GPU) and loads it."""
    from paper_2606_15991_gb300 import build, _lib

    build.build()
    return _lib.lib()


@pytest.fixture(scope="session")
def ctx(built_lib):
    import torch

    import paper_2606_15991_gb300 as tp

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = tp.tp_ctx_create(0)
    yield c
    torch.cuda.synchronize()
