import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels through the C ABI)")


def rel_err(x, ref):
    """Relative 2-norm error ||x - ref|| / ||ref||, the paper's measure (Sec. 5)."""
    import numpy as np

    x = np.asarray(x, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / (den if den > 0 else 1.0))


@pytest.fixture(scope="session")
def gm():
    """The CUDA library through its Python binding; skips when no GPU is present."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_06976_gb300 import gravmag

    gravmag.load()
    return gravmag
