import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def pytest_collection_modifyitems(config, items):
    # GPU tests cannot run without a device: skip them instead of failing when
    # collected on a CPU-only host without -m "not gpu".
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(scope="session")
def oracle():
    import oracle as _oracle
    _oracle._load()
    return _oracle


@pytest.fixture(autouse=True)
def _guard_bytes(request):
    """After every GPU test: no library buffer had its guard bytes changed
    (rgg_check_guards), i.e. nothing wrote past the end of a buffer."""
    yield
    if "gpu" not in request.keywords:
        return
    import torch
    if not torch.cuda.is_available():
        return
    from paper_2603_28674_gb300 import rgg
    checked, bad = rgg.check_guards()
    assert bad == 0, f"{bad} of {checked} library buffers had their guard bytes changed"
