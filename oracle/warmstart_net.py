"""CPU oracle of the learned warm-start network (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and nothing in the product
package.  The paper has no network (it leaves the inversion that uses its
operators to future work, Sec. 6); this module is the plain definition of the
network the library adds, written with PyTorch CPU ops in float64:

  encoder  E0 conv 1x3x3, 1 -> 32, ReLU; E1..E4 conv 1x3x3 with stride (1,2,2),
           32 -> 64 -> 128 -> 256 -> 512, ReLU          (S x S down to S/16)
  reshape  N x 512 x 1 x s x s -> N x 128 x 4 x s x s (row-major view: new
           channel c' and depth z come from old channel 4 c' + z)
  decoder  D1 nearest up-sampling (2,2,2) then conv 3x3x3 128 -> 64, ReLU;
           D2 up (2,2,2), 64 -> 32, ReLU; D3 up (1,2,2), 32 -> 16, ReLU;
           D4 up (1,2,2), 16 -> 1, no activation         (16 x S x S)
  net(d) = out_scale * f(in_scale * d)
  loss   = mean over all outputs of (f(in_scale d) - m / out_scale)^2
           [+ lam * mean over stations of (in_scale (G net(d) - d))^2, G dense]

Every convolution is a cross-correlation with "same" zero padding (1 in each
convolved axis) and a bias.  Parameters are one flat vector: per layer, in
the order above, w[co][ci][kd][kh][kw] then b[co].  The library convolves with
BF16 weights; ``bf16_round`` gives the same weights here (round to nearest
even of the FP32 value to 8 mantissa bits) so both sides use one set of
numbers.  Gradients are torch.autograd in float64.  The library's tensor-core kernels carry
the FP32 activations and gradients they multiply as two BF16 terms (hi + lo, relative error of
order 1e-6) and sum in FP32, which the default (exact operand) mode here models.  With
``bf16_operands=True`` the oracle instead rounds every convolution operand to a single BF16
value at the places a single-term BF16 GEMM would (its explicit backward formulas are pinned
against autograd with the rounding switched off).

Pins (tests/test_warmstart_oracle_pins.py): the convolution step against a
brute-force loop sum, the up-sampling and reshape against index formulas, the
parameter count, the gradient against central finite differences of the loss,
and Adam against its update rule written out for one scalar.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

# (in channels, out channels, kernel depth, in-plane stride, up-sampling (z, y, x), ReLU)
LAYERS = (
    (1, 32, 1, 1, (1, 1, 1), True),
    (32, 64, 1, 2, (1, 1, 1), True),
    (64, 128, 1, 2, (1, 1, 1), True),
    (128, 256, 1, 2, (1, 1, 1), True),
    (256, 512, 1, 2, (1, 1, 1), True),
    (128, 64, 3, 1, (2, 2, 2), True),
    (64, 32, 3, 1, (2, 2, 2), True),
    (32, 16, 3, 1, (1, 2, 2), True),
    (16, 1, 3, 1, (1, 2, 2), False),
)
DEPTH = 16


def num_params() -> int:
    return sum(co * ci * kd * 9 + co for ci, co, kd, _, _, _ in LAYERS)


def unpack(params):
    """Flat parameter vector -> list of (w [co, ci, kd, 3, 3], b [co]) float64 tensors."""
    p = torch.as_tensor(np.asarray(params, dtype=np.float64))
    out, off = [], 0
    for ci, co, kd, _, _, _ in LAYERS:
        nw = co * ci * kd * 9
        w = p[off:off + nw].reshape(co, ci, kd, 3, 3)
        off += nw
        b = p[off:off + co]
        off += co
        out.append((w, b))
    assert off == p.numel()
    return out


def bf16_round(x) -> np.ndarray:
    """Round FP32 values to the nearest BF16 value (ties to even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def conv_weights_bf16(params) -> np.ndarray:
    """The parameter vector with every convolution weight rounded to BF16, biases unchanged."""
    p = np.asarray(params, dtype=np.float64).copy()
    off = 0
    for ci, co, kd, _, _, _ in LAYERS:
        nw = co * ci * kd * 9
        p[off:off + nw] = bf16_round(p[off:off + nw])
        off += nw + co
    return p


def _round_bf16_tensor(t):
    return torch.as_tensor(bf16_round(t.detach().numpy()))


class _Bf16OperandConv(torch.autograd.Function):
    """A convolution whose operands are BF16 values, summed exactly (float64): the forward
    multiplies bf16(x) by the (already BF16) weights; the backward forms the data gradient from
    bf16(g) and the weights, the weight gradient from bf16(x) and bf16(g), and the bias gradient
    as the sum of bf16(g).  ``rounding=False`` leaves every operand as it is, which makes this
    the plain convolution and its exact gradient."""

    @staticmethod
    def forward(ctx, x, w, b, stride, pad, rounding):
        xr = _round_bf16_tensor(x) if rounding else x
        ctx.save_for_backward(xr, w)
        ctx.stride, ctx.pad, ctx.rounding = stride, pad, rounding
        return F.conv3d(xr, w, b, stride=stride, padding=pad)

    @staticmethod
    def backward(ctx, g):
        xr, w = ctx.saved_tensors
        gr = _round_bf16_tensor(g) if ctx.rounding else g
        dx = torch.nn.grad.conv3d_input(xr.shape, w, gr, stride=ctx.stride, padding=ctx.pad)
        dw = torch.nn.grad.conv3d_weight(xr, w.shape, gr, stride=ctx.stride, padding=ctx.pad)
        return dx, dw, gr.sum(dim=(0, 2, 3, 4)), None, None, None


def conv_bf16(mode, w, x=None, g=None, b=None, stride=1, in_shape=None, round_operands=True):
    """One convolution with BF16 weights, summed exactly (the three products of
    ``_Bf16OperandConv``): mode 0 conv(x, bf16(w)) + b; mode 1 the data gradient of shape
    in_shape from g; mode 2 (weight gradient from x and g, sum of g).  With round_operands the
    operands x and g are rounded to BF16 too; without, they enter as the given FP32 values."""
    wt = torch.as_tensor(bf16_round(np.asarray(w, dtype=np.float32)).reshape(np.shape(w)))
    kd = wt.shape[2]
    st, pad = (1, stride, stride), (kd // 2, 1, 1)

    def operand(a):
        a = np.asarray(a, dtype=np.float32)
        return torch.as_tensor((bf16_round(a) if round_operands else a.astype(np.float64)).reshape(np.shape(a)))

    if mode == 0:
        xr = operand(x)
        bt = None if b is None else torch.as_tensor(np.asarray(b, dtype=np.float64))
        return F.conv3d(xr, wt, bt, stride=st, padding=pad).numpy()
    gr = operand(g)
    if mode == 1:
        return torch.nn.grad.conv3d_input(tuple(in_shape), wt, gr, stride=st, padding=pad).numpy()
    xr = operand(x)
    dw = torch.nn.grad.conv3d_weight(xr, tuple(wt.shape), gr, stride=st, padding=pad)
    return dw.numpy(), gr.sum(dim=(0, 2, 3, 4)).numpy()


def upsample(x, f):
    """Nearest up-sampling of N x C x D x H x W by integer factors f = (fz, fy, fx)."""
    for axis, k in zip((2, 3, 4), f):
        if k > 1:
            x = torch.repeat_interleave(x, k, dim=axis)
    return x


def f_scaled(layers, d, in_scale, bf16_operands=False, explicit_backward=False, pre_acts=None):
    """f(in_scale d) for d of shape (N, S, S); returns (N, 16, S, S).

    bf16_operands: every convolution multiplies BF16-rounded operands (see _Bf16OperandConv);
    explicit_backward without it runs the same explicit gradient formulas with no rounding
    (used to pin them against autograd).  pre_acts, if a list, receives the input of every
    ReLU."""
    x = (in_scale * d).unsqueeze(1).unsqueeze(1)  # N x 1 x 1 x S x S
    for idx, ((ci, co, kd, st, up, relu), (w, b)) in enumerate(zip(LAYERS, layers)):
        if idx == 5:  # the encoder's 512 x 1 x s x s output read as 128 x 4 x s x s
            n, c, _, h, ww = x.shape
            x = x.reshape(n, c // 4, 4, h, ww)
        x = upsample(x, up)
        if bf16_operands or explicit_backward:
            x = _Bf16OperandConv.apply(x, w, b, (1, st, st), (kd // 2, 1, 1), bf16_operands)
        else:
            x = F.conv3d(x, w, b, stride=(1, st, st), padding=(kd // 2, 1, 1))
        if relu:
            if pre_acts is not None:
                pre_acts.append(x.detach())
            x = torch.relu(x)
    return x[:, 0]


def relu_margin(params, d, in_scale=1.0) -> float:
    """The smallest |input| of any ReLU of f(in_scale d), relative to the rms of its layer's
    inputs.  The gradient of the network jumps where a ReLU input crosses zero, so two
    evaluations that differ by a relative e per value agree to e only when this margin is well
    above e."""
    pre = []
    with torch.no_grad():
        f_scaled(unpack(params), torch.as_tensor(np.asarray(d, dtype=np.float64)), in_scale, pre_acts=pre)
    return min(float(x.abs().min() / torch.sqrt((x * x).mean())) for x in pre)


def forward(params, d, in_scale=1.0, out_scale=1.0, bf16_operands=False) -> np.ndarray:
    """net(d) with the given parameters (used as they are: round them first for BF16 parity)."""
    with torch.no_grad():
        y = f_scaled(unpack(params), torch.as_tensor(np.asarray(d, dtype=np.float64)), in_scale, bf16_operands)
    return (out_scale * y).numpy()


def _data_term(y, d, in_scale, out_scale, G):
    """mean over examples and stations of (in_scale (G m_pred - d))^2, m_pred = out_scale y, with G
    a dense (S*S) x (16*S*S) matrix in the layouts d[j][i] and m[r][q][p] (x fastest)."""
    Gt = torch.as_tensor(np.asarray(G, dtype=np.float64))
    mp = (out_scale * y).reshape(y.shape[0], -1)
    r = in_scale * (mp @ Gt.T - d.reshape(d.shape[0], -1))
    return (r ** 2).mean()


def loss_and_grad(params, d, m, in_scale=1.0, out_scale=1.0, G=None, lam=0.0, bf16_operands=False,
                  explicit_backward=False):
    """(loss, gradient with respect to the flat parameter vector), float64.  With G and lam > 0
    the loss adds lam times the data term of ``_data_term``; bf16_operands / explicit_backward as
    in ``f_scaled``."""
    p = torch.tensor(np.asarray(params, dtype=np.float64), requires_grad=True)
    layers, off = [], 0
    for ci, co, kd, _, _, _ in LAYERS:
        nw = co * ci * kd * 9
        layers.append((p[off:off + nw].reshape(co, ci, kd, 3, 3), p[off + nw:off + nw + co]))
        off += nw + co
    dt = torch.as_tensor(np.asarray(d, dtype=np.float64))
    y = f_scaled(layers, dt, in_scale, bf16_operands, explicit_backward)
    t = torch.as_tensor(np.asarray(m, dtype=np.float64)) / out_scale
    loss = ((y - t) ** 2).mean()
    if lam > 0:
        loss = loss + lam * _data_term(y, dt, in_scale, out_scale, G)
    loss.backward()
    return loss.item(), p.grad.numpy().copy()


def loss(params, d, m, in_scale=1.0, out_scale=1.0, G=None, lam=0.0, bf16_operands=False) -> float:
    with torch.no_grad():
        dt = torch.as_tensor(np.asarray(d, dtype=np.float64))
        y = f_scaled(unpack(params), dt, in_scale, bf16_operands)
        t = torch.as_tensor(np.asarray(m, dtype=np.float64)) / out_scale
        v = ((y - t) ** 2).mean()
        if lam > 0:
            v = v + lam * _data_term(y, dt, in_scale, out_scale, G)
        return float(v)


def adam(w, g, m1, m2, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam update (Kingma & Ba, Algorithm 1); step counts from 1."""
    m1 = b1 * m1 + (1 - b1) * g
    m2 = b2 * m2 + (1 - b2) * g * g
    mhat = m1 / (1 - b1 ** step)
    vhat = m2 / (1 - b2 ** step)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m1, m2
