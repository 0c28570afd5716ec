import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def d2ip():
    """The C-ABI binding; builds libd2ip.so first when it is missing (no fallback)."""
    from paper_2507_14046_gb300 import build
    import os
    if not os.path.exists(build.OUT):
        build.build()
    from paper_2507_14046_gb300 import binding
    return binding
