"""Products of a plan whose buffers reuse memory that another plan has just freed.

Every apply reads only what the set-up or an earlier kernel of the same product wrote, so a plan
built on memory left over from a plan of another precision (whose buffers hold values of another
layout) must give bit-identical products to a plan built first.  A kernel that reads its input
before the previous kernel has written it (for instance a load scheduled above the dependency
wait of a programmatic launch), or an uninitialised workspace, shows up here as a difference.
The kernels are deterministic, so the comparison is exact.
"""
import numpy as np
import pytest

from paper_1912_06976_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# gravity (real even spectra, one-warp row kernels) and magnetic (complex spectra), on the row
# and column ladders, two layers so that the forward's layer groups finish through the atomic count
CASES = [
    W.Workload("x512", W.GRAVITY, 256, 16, 2, 20.0, 25.0, 15.0, 0, 0, 55.0, 20.0),
    W.Workload("y160", W.MAGNETIC, 16, 80, 2, 20.0, 25.0, 15.0, 0, 0, 55.0, 20.0),
    W.Workload("pad", W.GRAVITY, 40, 30, 3, 25.0, 25.0, 20.0, 4, 3, 90.0, 0.0),
]
SEQUENCES = {
    "f64 after df64": (2, 1),
    "df64 after f64": (1, 2),
    "f64 after f32": (0, 1),
    "f32 after f64": (1, 0),
}


def _products(gm, w, prec):
    import torch

    dt = torch.float32 if prec == 0 else torch.float64
    m = W.random_vector(w.model_shape, 7)
    d = W.random_vector(w.data_shape, 8)
    op = gm.Operator.from_workload(w, precision=prec)
    try:
        f = op.forward(torch.as_tensor(m, dtype=dt, device="cuda")).cpu().numpy()
        t = op.transpose(torch.as_tensor(d, dtype=dt, device="cuda")).cpu().numpy()
        f2 = op.forward(torch.as_tensor(m, dtype=dt, device="cuda")).cpu().numpy()
    finally:
        op.close()
    return f, t, f2


@pytest.mark.parametrize("seq", list(SEQUENCES), ids=list(SEQUENCES))
@pytest.mark.parametrize("w", CASES, ids=[c.name for c in CASES])
def test_plan_on_reused_memory_gives_identical_products(gm, w, seq):
    first, second = SEQUENCES[seq]
    ref = _products(gm, w, second)
    for _ in range(3):
        _products(gm, w, first)
        got = _products(gm, w, second)
        for a, b, name in zip(got, ref, ("forward", "transpose", "second forward")):
            assert np.array_equal(a, b), (seq, name, float(np.abs(a - b).max()))
