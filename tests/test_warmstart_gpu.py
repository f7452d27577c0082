"""The warm-start network's tensor-core kernels against the float64 CPU oracle of the network.

Every convolution is a tcgen05 GEMM with BF16 weights and FP32 accumulation; the FP32
activations and gradients enter as two BF16 terms each (hi + lo), so the products are those of
the FP32 values to a relative 1e-6 (one convolution at a time against the oracle's exact
operands: tests/test_conv3d_tc_gpu.py, 1e-5).  The oracle here runs the network in float64 with
the same BF16 weights and exact activations and gradients.  Through the nine layers of the
forward pass and the eighteen products of a training step the differences stay at the level of
the FP32 sums and the two-term operands (a few 1e-6); the bounds are 1e-4 on outputs, on the
whole gradient and on the loss, and 1e-3 on every layer's weight and bias gradients.  An
indexing error gives O(1).

The gradient jumps where a ReLU input changes sign, so the gradient tests use inputs whose ReLU
inputs all clear zero by KINK_MARGIN of their layer's rms in the oracle (found by scanning input
seeds), about three times the spread of the per-value differences.  Without it a single ReLU
input within 1e-6 of zero takes opposite sides in the two computations and moves the gradients
upstream of it by ~1e-3 (observed on the 16 x 16 grid for one seed).
"""
import numpy as np
import pytest

from oracle import warmstart_net as N
from tests.conftest import assert_close, rel_err

pytestmark = pytest.mark.gpu
TOL_FWD = 1e-4
TOL_GRAD = 1e-4
TOL_LAYER = 1e-3
TOL_LOSS = 1e-4
KINK_MARGIN = 1e-5


@pytest.fixture(scope="module")
def ws(gm):
    from paper_1912_06976_gb300 import warmstart

    return warmstart


def _inputs(S, batch, seed):
    rng = np.random.default_rng((seed, 0x99))
    d = rng.standard_normal((batch, S, S)).astype(np.float32)
    m = (0.3 * rng.standard_normal((batch, 16, S, S))).astype(np.float32)
    return d, m


def _cuda(a):
    import torch

    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _kink_free_inputs(net, S, batch, in_scale, seed0, tries=80):
    """The first of _inputs(S, batch, seed0 + k) whose ReLU inputs all clear zero by KINK_MARGIN
    (relative to each layer's rms) in the oracle with the network's BF16 weights."""
    p = N.conv_weights_bf16(net.get_params())
    for seed in range(seed0, seed0 + tries):
        d, m = _inputs(S, batch, seed)
        if N.relu_margin(p, d.astype(np.float64), in_scale) > KINK_MARGIN:
            return d, m
    pytest.fail(f"no input of {tries} seeds clears the ReLU kinks by {KINK_MARGIN}")


def test_parameter_count(ws):
    net = ws.WarmStartNet(grid=32, max_batch=2, seed=0)
    assert net.num_params == N.num_params() == 1858849
    net.close()


@pytest.mark.parametrize("S,batch", [(16, 3), (32, 2), (64, 2)])
def test_forward_matches_oracle(ws, S, batch):
    net = ws.WarmStartNet(grid=S, max_batch=4, seed=7)
    net.set_scales(0.8, 1.7)
    d, _ = _inputs(S, batch, 1)
    got = net.forward(_cuda(d)).cpu().numpy()
    p = N.conv_weights_bf16(net.get_params())
    ref = N.forward(p, d.astype(np.float64), 0.8, 1.7)
    assert got.shape == (batch, 16, S, S)
    assert_close(got, ref, TOL_FWD)
    # gather + scale, 9 convolutions (up-sampling folded in), their split-K finishes, output scale
    assert 11 <= net.last_launch_count() <= 20
    net.close()


def _layer_slices():
    out, off = [], 0
    for ci, co, kd, _, _, _ in N.LAYERS:
        nw = co * ci * kd * 9
        out.append((slice(off, off + nw), slice(off + nw, off + nw + co)))
        off += nw + co
    return out


@pytest.mark.parametrize("S,batch", [(16, 3), (32, 1)])
def test_loss_and_gradient_match_oracle(ws, S, batch):
    net = ws.WarmStartNet(grid=S, max_batch=4, seed=3)
    net.set_scales(1.1, 0.6)
    d, m = _kink_free_inputs(net, S, batch, 1.1, 2)
    loss = net.train_step(_cuda(d), _cuda(m), 0.0)
    g = net.get_params("grad").astype(np.float64)
    p = N.conv_weights_bf16(net.get_params())
    ref_loss, ref_g = N.loss_and_grad(p, d.astype(np.float64), m.astype(np.float64), 1.1, 0.6)
    assert abs(loss - ref_loss) <= TOL_LOSS * ref_loss
    per_layer = [(rel_err(g[ws_], ref_g[ws_]), rel_err(g[bs], ref_g[bs])) for ws_, bs in _layer_slices()]
    assert rel_err(g, ref_g) < TOL_GRAD, per_layer
    assert max(max(e) for e in per_layer) < TOL_LAYER, per_layer  # every layer's weights and biases
    assert net.step == 0  # lr = 0: no Adam step
    net.close()


def test_adam_step_matches_oracle_rule(ws):
    S = 16
    net = ws.WarmStartNet(grid=S, max_batch=2, seed=5)
    d, m = _inputs(S, 2, 3)
    w0 = net.get_params().astype(np.float64)
    net.train_step(_cuda(d), _cuda(m), 1e-3)
    g = net.get_params("grad").astype(np.float64)
    w1, m1, m2 = N.adam(w0, g, np.zeros_like(w0), np.zeros_like(w0), 1, 1e-3)
    assert np.max(np.abs(net.get_params() - w1)) < 1e-6
    assert rel_err(net.get_params("adam_m"), m1) < 1e-6
    # second step from the library's own FP32 state
    w1g = net.get_params().astype(np.float64)
    m1g, m2g = net.get_params("adam_m").astype(np.float64), net.get_params("adam_v").astype(np.float64)
    net.train_step(_cuda(d), _cuda(m), 2e-3)
    g2 = net.get_params("grad").astype(np.float64)
    w2, _, _ = N.adam(w1g, g2, m1g, m2g, 2, 2e-3)
    assert np.max(np.abs(net.get_params() - w2)) < 1e-6
    assert net.step == 2
    net.close()


def test_indexed_batch_equals_explicit_batch(ws):
    import torch

    S = 32
    d, m = _inputs(S, 6, 4)
    idx = np.array([4, 1, 1, 5], dtype=np.int32)
    a = ws.WarmStartNet(grid=S, max_batch=4, seed=9)
    b = ws.WarmStartNet(grid=S, max_batch=4, seed=9)
    la = a.train_step(_cuda(d), _cuda(m), 1e-3, index=torch.as_tensor(idx).cuda())
    lb = b.train_step(_cuda(d[idx]), _cuda(m[idx]), 1e-3)
    assert la == lb
    assert np.array_equal(a.get_params(), b.get_params())
    a.close()
    b.close()


def test_out_of_range_index_is_reported_not_read(ws, gm):
    import torch

    S = 16
    d, m = _inputs(S, 2, 5)
    net = ws.WarmStartNet(grid=S, max_batch=2, seed=1)
    with pytest.raises(gm.GravMagError, match="outside"):
        net.train_step(_cuda(d), _cuda(m), 0.0, index=torch.as_tensor(np.array([0, 2], np.int32)).cuda())
    # the flag is cleared and the handle stays usable
    assert np.isfinite(net.train_step(_cuda(d), _cuda(m), 0.0))
    net.close()


def test_checkpoint_resume_continues_the_same_trajectory(ws, tmp_path):
    S = 16
    d, m = _inputs(S, 2, 6)
    a = ws.WarmStartNet(grid=S, max_batch=2, seed=2)
    a.set_scales(0.5, 2.0)
    for _ in range(3):
        a.train_step(_cuda(d), _cuda(m), 1e-3)
    path = str(tmp_path / "ckpt.npz")
    a.save(path)
    for _ in range(2):
        a.train_step(_cuda(d), _cuda(m), 1e-3)
    b = ws.WarmStartNet(grid=S, max_batch=2, seed=99)
    b.load(path)
    assert b.step == 3 and (b.in_scale, b.out_scale) == (0.5, 2.0)
    for _ in range(2):
        b.train_step(_cuda(d), _cuda(m), 1e-3)
    assert np.array_equal(a.get_params(), b.get_params())
    a.close()
    b.close()


def test_training_is_deterministic(ws):
    S = 32
    d, m = _inputs(S, 4, 7)
    runs = []
    for _ in range(2):
        net = ws.WarmStartNet(grid=S, max_batch=4, seed=4)
        losses = [net.train_step(_cuda(d), _cuda(m), 1e-3) for _ in range(3)]
        runs.append((losses, net.get_params()))
        net.close()
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1], runs[1][1])


def test_data_term_loss_and_gradient_match_oracle(ws, gm):
    """Training with the data-consistency term: the library's FP32 G / G^T inside the train step
    against the dense binary128 G of the prism oracle inside the float64 network oracle."""
    import oracle as O

    S = 16
    geom = O.Geometry.uniform(S, S, 16, 25.0, 25.0, 25.0)
    Gd = O.dense(geom)
    op = gm.Operator(S, S, 16, 25.0, 25.0, 25.0, precision=gm.F32)
    net = ws.WarmStartNet(grid=S, max_batch=4, seed=11)
    net.set_scales(0.3, 0.8)
    net.set_data_term(op, 0.5)
    d, m = _kink_free_inputs(net, S, 3, 0.3, 9)
    loss = net.train_step(_cuda(d), _cuda(m), 0.0)
    model_term, data_term = net.last_losses()
    g = net.get_params("grad").astype(np.float64)
    p = N.conv_weights_bf16(net.get_params())
    ref_loss, ref_g = N.loss_and_grad(p, d.astype(np.float64), m.astype(np.float64), 0.3, 0.8, Gd, 0.5)
    ref_model = N.loss(p, d.astype(np.float64), m.astype(np.float64), 0.3, 0.8)
    assert abs(model_term - ref_model) <= TOL_LOSS * ref_model
    assert abs(loss - ref_loss) <= TOL_LOSS * ref_loss
    assert abs(loss - (model_term + 0.5 * data_term)) <= 1e-6 * loss
    assert rel_err(g, ref_g) < TOL_GRAD, rel_err(g, ref_g)
    # lambda = 0 removes the term again
    net.set_data_term(None, 0.0)
    net.train_step(_cuda(d), _cuda(m), 0.0)
    assert net.last_losses()[1] == 0.0
    net.close()
    op.close()


def test_data_term_rejects_a_mismatched_operator(ws, gm):
    net = ws.WarmStartNet(grid=16, max_batch=2, seed=0)
    for op in (gm.Operator(16, 16, 16, 25.0, 25.0, 25.0, precision=gm.F64),
               gm.Operator(16, 16, 8, 25.0, 25.0, 25.0, precision=gm.F32),
               gm.Operator(16, 16, 16, 25.0, 25.0, 25.0, px=2, precision=gm.F32)):
        with pytest.raises(gm.GravMagError, match="operator"):
            net.set_data_term(op, 1.0)
        op.close()
    net.close()
