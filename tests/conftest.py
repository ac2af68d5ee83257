import os
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU check")


@pytest.fixture(autouse=True, scope="session")
def _oracle_threads():
    """Let the oracle use the host cores (it is deterministic for any thread count)."""
    try:
        import oracle
        oracle.set_threads(min(16, os.cpu_count() or 1))
    except Exception:
        pass
    yield
