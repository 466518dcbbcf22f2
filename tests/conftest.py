import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(scope="session")
def lib():
    """The CUDA library through its Python binding (GPU tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_00409_gb300 import psatd
    return psatd


@pytest.fixture
def metrics_log():
    """log(case, precision, rel_l2, tol): appends a parity record to the file
    named by $PSATD_METRICS_LOG (nothing when it is unset)."""
    from paper_2010_00409_gb300 import metrics
    path = os.environ.get(metrics.ENV)

    def log(case, precision, rel_l2, tol, **extra):
        if path:
            metrics.append(path, metrics.parity_record(case, precision, float(rel_l2), tol, **extra))
    return log
