import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    import warnings

    import numpy as np

    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels through the C ABI)")
    # a comparison that casts complex values to real drops their imaginary parts: fail instead
    complex_warning = getattr(getattr(np, "exceptions", np), "ComplexWarning")
    warnings.filterwarnings("error", category=complex_warning)


def _as_vector(a):
    import numpy as np

    a = np.asarray(a)
    return a.astype(np.complex128 if np.iscomplexobj(a) else np.float64).ravel()


def rel_err(x, ref):
    """Relative 2-norm error ||x - ref|| / ||ref||, the paper's measure (Sec. 5).  Complex
    inputs stay complex, so imaginary parts count."""
    import numpy as np

    x, ref = _as_vector(x), _as_vector(ref)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / (den if den > 0 else 1.0))


def max_err(x, ref):
    """Largest element error relative to the largest reference element, max|x - ref| / max|ref|:
    a few wrong outputs among many barely move the 2-norm but show here."""
    import numpy as np

    x, ref = _as_vector(x), _as_vector(ref)
    if x.size == 0:
        return 0.0
    den = float(np.max(np.abs(ref)))
    return float(np.max(np.abs(x - ref)) / (den if den > 0 else 1.0))


def assert_close(x, ref, tol, what=""):
    """The parity check: relative 2-norm error below tol and every element within tol of the
    largest reference element."""
    e2, einf = rel_err(x, ref), max_err(x, ref)
    assert e2 < tol and einf < tol, f"{what} rel 2-norm {e2:.3e}, max element {einf:.3e}, tol {tol:.0e}"


@pytest.fixture(scope="session")
def gm():
    """The CUDA library through its Python binding; skips when no GPU is present."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_06976_gb300 import gravmag

    gravmag.load()
    return gravmag
