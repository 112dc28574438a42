import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300) and the built libnuri.so")
    config.addinivalue_line("markers", "slow: long-running")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA GPU on this host")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(autouse=True)
def _query_time_budget(request):
    """Every query of a GPU test runs under a device time budget: a search that ran away
    fails its test with NURI_ERR_TIMEOUT (the message names the rounds and nodes it reached)
    instead of holding the run."""
    if "gpu" not in request.keywords:
        yield
        return
    import paper_1807_08888_b300 as nuri
    nuri.set_time_budget(120000.0)
    yield
    nuri.set_time_budget(0.0)

