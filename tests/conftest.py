import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the libiwpp CUDA library")
    config.addinivalue_line("markers", "slow: full-size workloads (minutes of oracle time)")


@pytest.fixture(scope="session")
def cuda_ctx():
    """A libiwpp context on cuda:0.  On a GPU test run the library must load:
    a missing build or missing GPU is a failure, not a skip."""
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1209_3314_gb300 import build

    build.build()
    from paper_1209_3314_gb300 import Context

    ctx = Context(0)
    yield ctx
    ctx.close()
