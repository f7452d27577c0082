"""Failure paths of the C ABI on a GPU, injected on the host (no kernel is made to fail):
a memory limit below a plan's need, overlapping buffers, NULL pointers and bad CGLS arguments.
Each must return its status before any device work or allocation, and leave a handle that
was valid before the failed call usable, with the same products as before."""
import ctypes

import numpy as np
import pytest

from paper_1912_06976_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _free_bytes():
    import torch

    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_memory_limit_gives_enomem_before_any_allocation(gm):
    """gm_set_memory_limit below the plan's need: GM_ENOMEM, nothing allocated (the paper's
    memory-safety test before a run, Sec. 6)."""
    w = W.WORKLOADS["mag64"]
    op = gm.Operator.from_workload(w, precision=gm.F32)  # warm up the library and its modules
    need = op.info.spectrum_bytes + op.info.workspace_bytes
    op.close()
    free0 = _free_bytes()
    gm.set_memory_limit(need // 2)
    try:
        with pytest.raises(gm.GravMagError) as e:
            gm.Operator.from_workload(w, precision=gm.F32)
        assert e.value.status == gm.GM_ENOMEM
        assert gm.load().gm_last_status() == gm.GM_ENOMEM
        assert _free_bytes() == free0
    finally:
        gm.set_memory_limit(0)
    op = gm.Operator.from_workload(w, precision=gm.F32)  # the limit lifted: set-up works again
    op.close()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_overlapping_buffers_are_einval_and_the_handle_stays_usable(gm, prec):
    import torch

    w = W.WORKLOADS["grav16"]
    op = gm.Operator.from_workload(w, precision=prec)
    lib = gm.load()
    dt = op.dtype
    m = torch.as_tensor(W.model("grav16"), dtype=dt, device="cuda").contiguous()
    d = torch.as_tensor(W.data("grav16"), dtype=dt, device="cuda").contiguous()
    ref_d = op.forward(m).clone()
    ref_m = op.transpose(d).clone()
    big = torch.zeros(op.info.n_model + op.info.n_data, dtype=dt, device="cuda")
    big[: op.info.n_model] = m.reshape(-1)
    es = big.element_size()
    base = big.data_ptr()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # output starting inside the input, input starting inside the output, the same buffer
    for a, b in ((base, base + es * 7), (base + es * 7, base), (base, base)):
        assert lib.apply_forward(op.handle, ctypes.c_void_p(a), ctypes.c_void_p(b), s) == gm.GM_EINVAL
        assert lib.apply_transpose(op.handle, ctypes.c_void_p(a), ctypes.c_void_p(b), s) == gm.GM_EINVAL
        assert lib.gm_last_status() == gm.GM_EINVAL
        assert b"overlap" in lib.gm_last_error()
    # NULL buffers and a NULL handle
    assert lib.apply_forward(op.handle, None, ctypes.c_void_p(d.data_ptr()), s) == gm.GM_EINVAL
    assert lib.apply_transpose(op.handle, ctypes.c_void_p(d.data_ptr()), None, s) == gm.GM_EINVAL
    assert lib.apply_forward(None, ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(d.data_ptr()), s) == gm.GM_EINVAL
    torch.cuda.synchronize()
    assert float(big[op.info.n_model:].abs().sum()) == 0.0  # no rejected call wrote anything
    # adjacent, non-overlapping buffers are accepted, and the handle gives the same products
    out_d = big[op.info.n_model:].view(op.data_shape)
    op.forward(big[: op.info.n_model].view(op.model_shape), out=out_d)
    assert torch.equal(out_d, ref_d)
    assert torch.equal(op.transpose(d), ref_m)
    op.close()


def test_bad_cgls_arguments_are_einval_and_the_handle_stays_usable(gm):
    import torch

    w = W.WORKLOADS["mag64"]
    op = gm.Operator.from_workload(w, precision=gm.F32)
    d = torch.as_tensor(W.data("mag64"), dtype=torch.float32, device="cuda")
    x_ref, res_ref = op.cgls(d, 1e-2, 5)
    out = torch.empty(op.model_shape, dtype=torch.float32, device="cuda")
    for alpha, iters in ((-1.0, 5), (float("nan"), 5), (1e-2, -1)):
        with pytest.raises(gm.GravMagError) as e:
            op.cgls(d, alpha, iters, out=out)
        assert e.value.status == gm.GM_EINVAL
        with pytest.raises(gm.GravMagError) as e:
            op.cgls_noalloc(d, alpha, iters, out)
        assert e.value.status == gm.GM_EINVAL
    x, res = op.cgls(d, 1e-2, 5)
    assert torch.equal(x, x_ref)
    np.testing.assert_array_equal(res, res_ref)
    op.close()


def test_status_strings_name_every_code(gm):
    lib = gm.load()
    for code, name in ((gm.GM_OK, b"GM_OK"), (gm.GM_EINVAL, b"GM_EINVAL"), (gm.GM_ENOMEM, b"GM_ENOMEM")):
        assert lib.gm_status_string(code).startswith(name)
