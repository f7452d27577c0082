"""The warm-start network's CUDA kernels against the float64 CPU oracle of the same network.

The library convolves with BF16 copies of its FP32 weights and accumulates in FP32; the oracle
is handed the same BF16-rounded weights, so what remains is FP32 rounding in sums of up to
27 * 128 products: outputs and gradients agree to a relative 2-norm error of 1e-4 (ReLU
decisions near zero may flip between the two precisions; each flip moves the result by a
value of the size of that rounding).
"""
import numpy as np
import pytest

from oracle import warmstart_net as N
from tests.conftest import rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-4


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
    assert rel_err(got, ref) < TOL
    assert net.last_launch_count() == 1 + 9 + 4 + 1  # gather+scale, 9 convs, 4 up-samplings, output scale
    net.close()


def _layer_slices():
    out, off = [], 0
    for ci, co, kd, _, _, _ in N.LAYERS:
        nw = co * ci * kd * 9
        out.append((slice(off, off + nw), slice(off + nw, off + nw + co)))
        off += nw + co
    return out


@pytest.mark.parametrize("S", [16, 32])
def test_loss_and_gradient_match_oracle(ws, S):
    net = ws.WarmStartNet(grid=S, max_batch=4, seed=3)
    net.set_scales(1.1, 0.6)
    d, m = _inputs(S, 3, 2)
    loss = net.train_step(_cuda(d), _cuda(m), 0.0)
    g = net.get_params("grad").astype(np.float64)
    p = N.conv_weights_bf16(net.get_params())
    ref_loss, ref_g = N.loss_and_grad(p, d.astype(np.float64), m.astype(np.float64), 1.1, 0.6)
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    per_layer = [(rel_err(g[ws_], ref_g[ws_]), rel_err(g[bs], ref_g[bs])) for ws_, bs in _layer_slices()]
    assert rel_err(g, ref_g) < TOL, per_layer
    assert max(max(e) for e in per_layer) < 10 * TOL, per_layer  # every layer's weights and biases
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
    against the dense long-double G of the prism oracle inside the float64 network oracle."""
    import oracle as O

    S = 16
    geom = O.Geometry.uniform(S, S, 16, 25.0, 25.0, 25.0)
    Gd = O.dense(geom)
    op = gm.Operator(S, S, 16, 25.0, 25.0, 25.0, precision=gm.F32)
    net = ws.WarmStartNet(grid=S, max_batch=4, seed=11)
    net.set_scales(0.3, 0.8)
    net.set_data_term(op, 0.5)
    d, m = _inputs(S, 3, 9)
    loss = net.train_step(_cuda(d), _cuda(m), 0.0)
    model_term, data_term = net.last_losses()
    g = net.get_params("grad").astype(np.float64)
    p = N.conv_weights_bf16(net.get_params())
    ref_loss, ref_g = N.loss_and_grad(p, d.astype(np.float64), m.astype(np.float64), 0.3, 0.8, Gd, 0.5)
    ref_model = N.loss(p, d.astype(np.float64), m.astype(np.float64), 0.3, 0.8)
    assert abs(model_term - ref_model) <= 1e-5 * ref_model
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    assert abs(loss - (model_term + 0.5 * data_term)) <= 1e-6 * loss
    assert rel_err(g, ref_g) < TOL
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
