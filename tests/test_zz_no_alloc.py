"""The allocation-free CGLS entry point (gm_cgls_noalloc) against the regular one (gm_cgls).

gm_cgls_noalloc serves callers that cannot call cudaMalloc when they solve:
processes whose GPU memory a framework's pooling allocator has already
reserved, latency-critical loops that cannot take the device-wide
synchronisation an allocation may cause, and services that must not grow their
device footprint after start-up.  Its scratch is a fixed array inside the
library, shared by all calls, so these tests check that two calls in a row --
the second one seeing the first one's leftovers -- each give the same result
as gm_cgls in every precision (FP32, FP64 and double-float, whose vectors are
FP64), that the device's free memory is the same before and after each call,
and that a grid too large for the array is refused with a clear error.  This file is collected last so that a stop-at-first-failure run has
already run every other test.
"""
import numpy as np
import pytest

from paper_1912_06976_gb300 import workloads as W
from tests.conftest import assert_close, rel_err

pytestmark = pytest.mark.gpu

TOL = {1: 1e-12, 0: 1e-5, 2: 1e-12}


def _free_bytes():
    import torch

    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("prec", [1, 0, 2])
def test_noalloc_cgls_matches_cgls_twice_in_a_row(gm, prec):
    import torch

    w = W.WORKLOADS["mag64"]
    op = gm.Operator.from_workload(w, precision=prec)
    dt = op.dtype
    runs = [(W.data("mag64", 0), 1e-2, 12, None), (W.data("mag64", 1), 3e-2, 7, W.random_vector(w.model_shape, 5))]
    for d_np, alpha, iters, x0_np in runs:
        d = torch.as_tensor(d_np, dtype=dt, device="cuda")
        x0 = torch.as_tensor(x0_np, dtype=dt, device="cuda") if x0_np is not None else None
        ref, ref_res = op.cgls(d, alpha, iters, x0=x0)
        out = torch.empty(op.model_shape, dtype=dt, device="cuda")
        free0 = _free_bytes()
        got, got_res = op.cgls_noalloc(d, alpha, iters, out, x0=x0)
        assert _free_bytes() == free0  # the call allocated no device memory
        assert got.data_ptr() == out.data_ptr()
        assert_close(got.double().cpu().numpy(), ref.double().cpu().numpy(), TOL[prec])
        np.testing.assert_allclose(got_res, ref_res, rtol=TOL[prec])
    op.close()


def test_noalloc_cgls_rejects_grids_beyond_its_array(gm):
    import torch

    op = gm.Operator(200, 200, 60, 10.0, 10.0, 10.0, precision=gm.F32)  # (2n + 2m) * 4 B > 16 MiB
    cap = gm.load().gm_cgls_noalloc_capacity()
    assert cap == 16 << 20
    d = torch.zeros(op.data_shape, dtype=torch.float32, device="cuda")
    out = torch.empty(op.model_shape, dtype=torch.float32, device="cuda")
    with pytest.raises(gm.GravMagError) as e:
        op.cgls_noalloc(d, 1e-2, 5, out)
    assert e.value.status == gm.GM_EINVAL
    assert "fixed array" in str(e.value)
    op.close()
