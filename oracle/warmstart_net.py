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
numbers.  Gradients are torch.autograd in float64.

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


def upsample(x, f):
    """Nearest up-sampling of N x C x D x H x W by integer factors f = (fz, fy, fx)."""
    for axis, k in zip((2, 3, 4), f):
        if k > 1:
            x = torch.repeat_interleave(x, k, dim=axis)
    return x


def f_scaled(layers, d, in_scale):
    """f(in_scale d) for d of shape (N, S, S); returns (N, 16, S, S)."""
    x = (in_scale * d).unsqueeze(1).unsqueeze(1)  # N x 1 x 1 x S x S
    for idx, ((ci, co, kd, st, up, relu), (w, b)) in enumerate(zip(LAYERS, layers)):
        if idx == 5:  # the encoder's 512 x 1 x s x s output read as 128 x 4 x s x s
            n, c, _, h, ww = x.shape
            x = x.reshape(n, c // 4, 4, h, ww)
        x = upsample(x, up)
        x = F.conv3d(x, w, b, stride=(1, st, st), padding=(kd // 2, 1, 1))
        if relu:
            x = torch.relu(x)
    return x[:, 0]


def forward(params, d, in_scale=1.0, out_scale=1.0) -> np.ndarray:
    """net(d) with the given parameters (used as they are: round them first for BF16 parity)."""
    with torch.no_grad():
        y = f_scaled(unpack(params), torch.as_tensor(np.asarray(d, dtype=np.float64)), in_scale)
    return (out_scale * y).numpy()


def _data_term(y, d, in_scale, out_scale, G):
    """mean over examples and stations of (in_scale (G m_pred - d))^2, m_pred = out_scale y, with G
    a dense (S*S) x (16*S*S) matrix in the layouts d[j][i] and m[r][q][p] (x fastest)."""
    Gt = torch.as_tensor(np.asarray(G, dtype=np.float64))
    mp = (out_scale * y).reshape(y.shape[0], -1)
    r = in_scale * (mp @ Gt.T - d.reshape(d.shape[0], -1))
    return (r ** 2).mean()


def loss_and_grad(params, d, m, in_scale=1.0, out_scale=1.0, G=None, lam=0.0):
    """(loss, gradient with respect to the flat parameter vector), float64.  With G and lam > 0
    the loss adds lam times the data term of ``_data_term``."""
    p = torch.tensor(np.asarray(params, dtype=np.float64), requires_grad=True)
    layers, off = [], 0
    for ci, co, kd, _, _, _ in LAYERS:
        nw = co * ci * kd * 9
        layers.append((p[off:off + nw].reshape(co, ci, kd, 3, 3), p[off + nw:off + nw + co]))
        off += nw + co
    dt = torch.as_tensor(np.asarray(d, dtype=np.float64))
    y = f_scaled(layers, dt, in_scale)
    t = torch.as_tensor(np.asarray(m, dtype=np.float64)) / out_scale
    loss = ((y - t) ** 2).mean()
    if lam > 0:
        loss = loss + lam * _data_term(y, dt, in_scale, out_scale, G)
    loss.backward()
    return loss.item(), p.grad.numpy().copy()


def loss(params, d, m, in_scale=1.0, out_scale=1.0, G=None, lam=0.0) -> float:
    with torch.no_grad():
        dt = torch.as_tensor(np.asarray(d, dtype=np.float64))
        y = f_scaled(unpack(params), dt, in_scale)
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
