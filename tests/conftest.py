import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libst.so")
    config.addinivalue_line("markers", "slow: full-size case, takes longer than a few seconds")


@pytest.fixture(autouse=True)
def _gpu_required(request):
    """GPU-marked tests fail (never skip) when CUDA or the library is absent."""
    if request.node.get_closest_marker("gpu") is None:
        return
    import torch

    if not torch.cuda.is_available():
        pytest.fail("test marked gpu but torch.cuda.is_available() is False")
    import paper_1912_10082_gb300 as st

    st.lib()
