"""The tensor-core convolution kernels one at a time (gm_conv3d) against the oracle's
convolution of the exact FP32 operands with BF16 weights, summed exactly in float64.

The kernels carry each FP32 activation and gradient as two BF16 terms (hi + lo: rms relative
representation error about 1.3e-6) and accumulate the products in FP32 over K = 9 or 27 taps x
up to 512 channels (or over all positions for the weight gradient, whose lo x lo term is left
out, about 1.3e-6 of each product): a relative 2-norm error of order 2e-6; the bound is 1e-5.  The geometries
cover one input channel, one output channel (on the tensor cores for few (sample, plane) pairs,
on the CUDA-core kernels for many), odd sizes that leave ragged 128-row tiles, stride 2, 3-D
kernels and two 256-column tiles.
"""
import numpy as np
import pytest

from oracle import warmstart_net as N
from tests.conftest import assert_close, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-5

# (batch, CI, CO, D, H, W, KD, stride)
GEOMS = [
    (2, 1, 32, 1, 16, 16, 1, 1),
    (3, 32, 64, 1, 17, 15, 1, 2),
    (1, 256, 512, 1, 8, 8, 1, 2),
    (2, 128, 64, 8, 6, 6, 3, 1),
    (2, 16, 1, 5, 9, 7, 3, 1),
    (1, 64, 32, 4, 5, 3, 3, 1),
    (2, 8, 16, 3, 33, 31, 3, 2),
    # one output channel with enough (sample, plane) pairs that every mode takes the CUDA-core kernels
    (20, 16, 1, 16, 12, 21, 3, 1),
    (24, 4, 1, 13, 7, 33, 1, 1),
]


def _data(geom, seed):
    n, ci, co, d, h, w, kd, st = geom
    rng = np.random.default_rng((seed, 0xC0))
    oh, ow = (h - 1) // st + 1, (w - 1) // st + 1
    x = rng.standard_normal((n, ci, d, h, w)).astype(np.float32)
    g = rng.standard_normal((n, co, d, oh, ow)).astype(np.float32)
    wt = (rng.standard_normal((co, ci, kd, 3, 3)) / np.sqrt(ci * kd * 9)).astype(np.float32)
    b = rng.standard_normal(co).astype(np.float32)
    return x, g, wt, b


def _cuda(a):
    import torch

    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def ws(gm):
    from paper_1912_06976_gb300 import warmstart

    return warmstart


@pytest.mark.parametrize("geom", GEOMS, ids=[f"n{g[0]}c{g[1]}k{g[2]}d{g[3]}h{g[4]}w{g[5]}kd{g[6]}s{g[7]}" for g in GEOMS])
def test_conv_modes_match_bf16_operand_oracle(ws, geom):
    import torch

    x, g, w, b = _data(geom, 1)
    st = geom[7]
    out = ws.conv3d(0, _cuda(w), x=_cuda(x), b=_cuda(b), stride=st).cpu().numpy()
    assert rel_err(out, N.conv_bf16(0, w, x=x, b=b, stride=st, round_operands=False)) < TOL
    dx = torch.empty(x.shape, dtype=torch.float32, device="cuda")
    ws.conv3d(1, _cuda(w), g=_cuda(g), stride=st, out=dx)
    assert rel_err(dx.cpu().numpy(), N.conv_bf16(1, w, g=g, stride=st, in_shape=x.shape, round_operands=False)) < TOL
    db = torch.empty(geom[2], dtype=torch.float32, device="cuda")
    dw = ws.conv3d(2, _cuda(w), x=_cuda(x), g=_cuda(g), stride=st, bias_grad=db).cpu().numpy()
    ref_w, ref_b = N.conv_bf16(2, w, x=x, g=g, stride=st, round_operands=False)
    assert rel_err(dw, ref_w) < TOL
    assert rel_err(db.cpu().numpy(), ref_b) < TOL


def test_conv_without_bias_and_bad_arguments(ws, gm):
    import torch

    x, g, w, b = _data(GEOMS[1], 2)
    out = ws.conv3d(0, _cuda(w), x=_cuda(x), stride=2).cpu().numpy()
    assert rel_err(out, N.conv_bf16(0, w, x=x, stride=2, round_operands=False)) < TOL
    w3 = torch.zeros((64, 24, 1, 3, 3), device="cuda")  # 24 input channels: not a power of two
    with pytest.raises(gm.GravMagError, match="powers of two"):
        ws.conv3d(0, w3, x=torch.zeros((1, 24, 1, 8, 8), device="cuda"))
