import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (runs the sm_103a library)")
    config.addinivalue_line(
        "markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def oracle():
    import oracle as _oracle
    _oracle.build()
    return _oracle


def pytest_collection_finish(session):
    """Start the background oracle solves of the full-size parity tests as
    soon as the session is known to run them (on a machine with a GPU)."""
    if not any("test_gpu_fullsize.py" in item.nodeid for item in session.items):
        return
    try:
        import torch
        if not torch.cuda.is_available():
            return
    except Exception:
        return
    import oracle_jobs
    oracle_jobs.start()


def pytest_sessionfinish(session, exitstatus):
    import sys
    mod = sys.modules.get("oracle_jobs")
    if mod is not None:
        mod.shutdown()
