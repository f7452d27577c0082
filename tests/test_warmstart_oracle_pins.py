"""Pins of the warm-start network oracle against definitions that do not go through it."""
import itertools

import numpy as np
import pytest
import torch

from oracle import warmstart_net as N


def brute_conv(x, w, b, stride, pad):
    """Cross-correlation by explicit loops: out[co, o] = b[co] + sum w[co, ci, t] x[ci, o*s + t - p]."""
    ci_, d, h, wd = x.shape
    co_, _, kd, kh, kw = w.shape
    od = (d + 2 * pad[0] - kd) // stride[0] + 1
    oh = (h + 2 * pad[1] - kh) // stride[1] + 1
    ow = (wd + 2 * pad[2] - kw) // stride[2] + 1
    out = np.zeros((co_, od, oh, ow))
    for co, z, y, xx in itertools.product(range(co_), range(od), range(oh), range(ow)):
        s = b[co]
        for ci, a, c, e in itertools.product(range(ci_), range(kd), range(kh), range(kw)):
            iz, iy, ix = z * stride[0] + a - pad[0], y * stride[1] + c - pad[1], xx * stride[2] + e - pad[2]
            if 0 <= iz < d and 0 <= iy < h and 0 <= ix < wd:
                s += w[co, ci, a, c, e] * x[ci, iz, iy, ix]
        out[co, z, y, xx] = s
    return out


@pytest.mark.parametrize("stride,kd", [((1, 1, 1), 3), ((1, 2, 2), 1), ((1, 2, 2), 3)])
def test_library_conv_is_the_loop_sum(stride, kd):
    """The conv3d call the oracle uses is the cross-correlation with the stated padding/stride."""
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 4, 7, 6))
    w = rng.standard_normal((3, 2, kd, 3, 3))
    b = rng.standard_normal(3)
    pad = (kd // 2, 1, 1)
    got = torch.nn.functional.conv3d(torch.as_tensor(x)[None], torch.as_tensor(w), torch.as_tensor(b),
                                     stride=stride, padding=pad)[0].numpy()
    assert np.allclose(got, brute_conv(x, w, b, stride, pad), rtol=0, atol=1e-12)


def test_upsample_index_formula():
    x = torch.arange(2 * 3 * 2 * 3 * 4, dtype=torch.float64).reshape(2, 3, 2, 3, 4)
    y = N.upsample(x, (2, 3, 2))
    for n, c, z, yy, xx in itertools.product(range(2), range(3), range(4), range(9), range(8)):
        assert y[n, c, z, yy, xx] == x[n, c, z // 2, yy // 3, xx // 2]


def test_parameter_count_and_layout():
    assert N.num_params() == 1858849
    p = np.arange(N.num_params(), dtype=np.float64)
    layers = N.unpack(p)
    assert layers[0][0].shape == (32, 1, 1, 3, 3) and layers[0][1][0] == 32 * 9
    assert layers[-1][0].shape == (1, 16, 3, 3, 3) and layers[-1][1][0] == N.num_params() - 1


def test_shapes_and_reshape_convention():
    """Output shape (N, 16, S, S); the decoder's first input depth z of channel c' is encoder
    channel 4 c' + z: a network whose encoder output is a known channel ramp shows it."""
    S = 16
    rng = np.random.default_rng(0)
    p = rng.standard_normal(N.num_params()) * 0.05
    out = N.forward(p, rng.standard_normal((2, S, S)))
    assert out.shape == (2, 16, S, S)
    x = torch.arange(512, dtype=torch.float64).reshape(1, 512, 1, 1, 1)
    v = x.reshape(1, 128, 4, 1, 1)
    for c in (0, 5, 127):
        for z in range(4):
            assert v[0, c, z, 0, 0] == 4 * c + z


def test_bf16_round_known_values():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 1.0 + 2 ** -9, -3.140625, 1e-40], dtype=np.float32)
    got = N.bf16_round(vals)
    # 1 + 2^-8: tie between 1 and 1 + 2^-7 -> even (1); 1 + 3*2^-9 above the tie -> 1 + 2^-7
    assert got[0] == 1.0 and got[1] == 1.0 and got[2] == 1.0 + 2 ** -7 and got[3] == 1.0
    assert got[4] == -3.140625
    assert got[5] == 2.0 ** -133  # subnormal: 0x000116C2 rounds down to 0x00010000


def test_gradient_matches_finite_differences():
    """Central differences of the float64 loss along random directions (S = 16, batch 2)."""
    S = 16
    rng = np.random.default_rng(3)
    p = rng.standard_normal(N.num_params()) * 0.05
    d = rng.standard_normal((2, S, S))
    m = rng.standard_normal((2, 16, S, S))
    loss, g = N.loss_and_grad(p, d, m, 0.7, 1.3)
    assert abs(loss - N.loss(p, d, m, 0.7, 1.3)) < 1e-14 * abs(loss)
    h = 1e-5
    for k in range(4):
        v = np.random.default_rng((k, 9)).standard_normal(p.size)
        v /= np.linalg.norm(v)
        fd = (N.loss(p + h * v, d, m, 0.7, 1.3) - N.loss(p - h * v, d, m, 0.7, 1.3)) / (2 * h)
        assert abs(fd - g @ v) <= 1e-6 * max(abs(fd), np.linalg.norm(g) * 1e-3)


def test_gradient_of_single_weights_by_differences():
    """Individual weights of the first, the middle (reshape-crossing) and the last layer."""
    S = 16
    rng = np.random.default_rng(4)
    p = rng.standard_normal(N.num_params()) * 0.05
    d = rng.standard_normal((1, S, S))
    m = rng.standard_normal((1, 16, S, S))
    _, g = N.loss_and_grad(p, d, m)
    offs = np.cumsum([0] + [co * ci * kd * 9 + co for ci, co, kd, _, _, _ in N.LAYERS])
    for idx in (3, offs[5] + 17, offs[8] + 5, offs[9] - 1):
        e = np.zeros_like(p)
        e[idx] = 1e-5
        fd = (N.loss(p + e, d, m) - N.loss(p - e, d, m)) / 2e-5
        assert abs(fd - g[idx]) <= 1e-6 * max(abs(fd), 1e-6)


def test_adam_matches_scalar_rule():
    w, g = np.array([0.5]), np.array([0.2])
    m1 = np.zeros(1)
    m2 = np.zeros(1)
    w1, m1, m2 = N.adam(w, g, m1, m2, 1, 0.01)
    # first step: mhat = g, vhat = g^2, update lr * g / (|g| + eps)
    assert np.allclose(w1, 0.5 - 0.01 * 0.2 / (0.2 + 1e-8), rtol=0, atol=1e-15)
    w2, _, _ = N.adam(w1, np.array([-0.1]), m1, m2, 2, 0.01)
    a = 0.9 * 0.1 * 0.2 + 0.1 * -0.1
    v = 0.999 * 0.001 * 0.04 + 0.001 * 0.01
    assert np.allclose(w2, w1 - 0.01 * (a / (1 - 0.81)) / (np.sqrt(v / (1 - 0.999 ** 2)) + 1e-8), rtol=0,
                       atol=1e-15)


def test_data_term_gradient_matches_finite_differences():
    """The loss with the data-consistency term, G a random dense matrix (S = 16)."""
    S = 16
    rng = np.random.default_rng(8)
    p = rng.standard_normal(N.num_params()) * 0.05
    d = rng.standard_normal((2, S, S))
    m = rng.standard_normal((2, 16, S, S))
    G = rng.standard_normal((S * S, 16 * S * S)) / 64.0
    loss, g = N.loss_and_grad(p, d, m, 0.9, 1.2, G, 0.7)
    assert abs(loss - N.loss(p, d, m, 0.9, 1.2, G, 0.7)) < 1e-14 * abs(loss)
    assert loss > N.loss(p, d, m, 0.9, 1.2)  # the term is added, and positive
    h = 1e-5
    for k in range(3):
        v = np.random.default_rng((k, 10)).standard_normal(p.size)
        v /= np.linalg.norm(v)
        fd = (N.loss(p + h * v, d, m, 0.9, 1.2, G, 0.7) - N.loss(p - h * v, d, m, 0.9, 1.2, G, 0.7)) / (2 * h)
        assert abs(fd - g @ v) <= 1e-6 * max(abs(fd), np.linalg.norm(g) * 1e-3)


def test_data_term_of_an_exact_model_is_zero():
    """If net(d) reproduces a model whose data are d, the data term vanishes: a network whose last
    layer is zero predicts its bias, so G applied to that constant model gives d exactly."""
    S = 16
    p = np.zeros(N.num_params())
    p[-1] = 0.25  # bias of the output layer: f = 0.25 everywhere
    G = np.random.default_rng(2).standard_normal((S * S, 16 * S * S))
    mp = np.full(16 * S * S, 0.25 * 1.5)
    d = (G @ mp).reshape(1, S, S)
    base = N.loss(p, d, np.zeros((1, 16, S, S)), 1.0, 1.5)
    assert abs(N.loss(p, d, np.zeros((1, 16, S, S)), 1.0, 1.5, G, 3.0) - base) < 1e-20 + 1e-12 * base


def test_explicit_backward_formulas_equal_autograd():
    """The explicit data / weight / bias gradient formulas of the BF16-operand convolution, with
    the rounding switched off, reproduce autograd's gradient of the plain network."""
    S = 16
    rng = np.random.default_rng(12)
    p = rng.standard_normal(N.num_params()) * 0.05
    d = rng.standard_normal((2, S, S))
    m = rng.standard_normal((2, 16, S, S))
    l1, g1 = N.loss_and_grad(p, d, m, 0.8, 1.1)
    l2, g2 = N.loss_and_grad(p, d, m, 0.8, 1.1, explicit_backward=True)
    assert abs(l1 - l2) <= 1e-15 * abs(l1)
    assert np.linalg.norm(g1 - g2) <= 1e-13 * np.linalg.norm(g1)


def test_bf16_operand_forward_is_conv_of_rounded_operands():
    """With BF16 operands, the first layer's output is the loop-sum convolution of the rounded
    input (the weights are passed already rounded)."""
    S = 16
    rng = np.random.default_rng(13)
    p = N.conv_weights_bf16(rng.standard_normal(N.num_params()) * 0.05)
    d = rng.standard_normal((1, S, S))
    (w, b), = N.unpack(p)[:1]
    x = torch.as_tensor(d).reshape(1, 1, 1, S, S)
    y = N._Bf16OperandConv.apply(x, w, b, (1, 1, 1), (0, 1, 1), True)
    xr = N.bf16_round(d).reshape(1, 1, S, S)
    ref = brute_conv(xr, w.numpy(), b.numpy(), (1, 1, 1), (0, 1, 1))
    assert np.allclose(y[0].numpy(), ref, rtol=0, atol=1e-12)
    # and the rounding is visible: the unrounded input gives a different result
    assert not np.allclose(y[0].numpy(), brute_conv(d.reshape(1, 1, S, S), w.numpy(), b.numpy(), (1, 1, 1),
                                                    (0, 1, 1)), rtol=0, atol=1e-9)


def test_bf16_operand_gradient_is_close_to_the_exact_one():
    """Rounding the GEMM operands to BF16 changes the gradient by a few percent (the BF16 unit
    2^-8 per operand, compounded over the 18 products of the forward and backward passes)."""
    S = 16
    rng = np.random.default_rng(14)
    p = N.conv_weights_bf16(rng.standard_normal(N.num_params()) * 0.05)
    d = rng.standard_normal((2, S, S))
    m = rng.standard_normal((2, 16, S, S))
    _, g1 = N.loss_and_grad(p, d, m)
    _, g2 = N.loss_and_grad(p, d, m, bf16_operands=True)
    rel = np.linalg.norm(g1 - g2) / np.linalg.norm(g1)
    assert 1e-4 < rel < 1e-1


def test_relu_margin_is_the_smallest_relu_input_over_its_layer_rms():
    """With all weights zero every ReLU input equals its channel's bias at every position, so
    the margin is min over ReLU layers of min_c |b_c| / sqrt(mean_c b_c^2) (each channel has the
    same number of positions); layer 3 gets one small bias, which must set the margin."""
    p = np.zeros(N.num_params())
    off, expect = 0, []
    for li, (ci, co, kd, _, _, relu) in enumerate(N.LAYERS):
        off += co * ci * kd * 9
        b = 0.5 + np.arange(co, dtype=np.float64) / co
        if li == 3:
            b[7] = 0.003
        p[off:off + co] = b
        off += co
        if relu:
            expect.append(np.min(np.abs(b)) / np.sqrt(np.mean(b * b)))
    d = np.random.default_rng(0).standard_normal((2, 16, 16))
    got = N.relu_margin(p, d)
    assert got == pytest.approx(min(expect), rel=1e-12)
    assert int(np.argmin(expect)) == 3  # the small bias of layer 3 sets it
