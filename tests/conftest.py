import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (sm_103a) and the built libne.so")


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle as o
    o.build()
    return o


@pytest.fixture(autouse=True)
def _index_status_clear(request):
    """Under the debug build (NE_INDEX_CHECKS=1), a GPU test must end with
    no index-check violation recorded by any kernel it launched."""
    if os.environ.get("NE_INDEX_CHECKS") != "1" or \
            request.node.get_closest_marker("gpu") is None:
        yield
        return
    import torch
    if not torch.cuda.is_available():
        yield
        return
    from paper_1509_03838_gb300 import ne
    ne.ne_debug_index_status(clear=True)
    yield
    v, first = ne.ne_debug_index_status(clear=True)
    assert v == 0, (f"{v} index-check violations; first at site {first >> 48}, "
                    f"index {first & ((1 << 48) - 1)}")
