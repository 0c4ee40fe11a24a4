import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: full-size case (minutes of CPU oracle time)")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def built_lib():
    """Path of the CUDA library, building it in-tree when missing."""
    from paper_2603_20481_gb300 import build
    return build.build(checked=os.environ.get("RISE_CHECKED") == "1")


@pytest.fixture(scope="session")
def det(built_lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_20481_gb300 import rise
    d = rise.Detector(0)
    yield d
    d.close()
