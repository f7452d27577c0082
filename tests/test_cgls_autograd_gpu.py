"""Differentiation and inversion on top of the fast operator (GPU).

* The autograd Function's backward is the transpose product: its gradient of
  L(m) = 1/2 ||G m - d||^2 is checked against central finite differences of L
  evaluated with the FP64 operator on 32 random directions, and the FP32
  dot-product test holds to 1e-6 (128 x 128 x 32 magnetic grid, I = 60, D = 0).
* CGLS on the device (FP64 and double-float handles) converges to the Tikhonov
  solution (G^T G + alpha^2 I)^-1 G^T d computed densely from oracle entries, and on the
  128 x 128 x 32 grid its reported residuals match ||G x_k - d|| recomputed.
"""
import numpy as np
import pytest

import oracle as O
from paper_1912_06976_gb300 import workloads as W
from tests.conftest import rel_err

pytestmark = pytest.mark.gpu


def _mag128_problem(gm):
    import torch

    w = W.WORKLOADS["mag128"]
    op32 = gm.Operator.from_workload(w, precision=gm.F32)
    op64 = gm.Operator.from_workload(w, precision=gm.F64)
    m_true = torch.as_tensor(W.model("mag128", 0), device="cuda")
    d_clean = op64.forward(m_true)
    d = d_clean + torch.as_tensor(W.noise(d_clean.cpu().numpy(), 0.01, 1), device="cuda")
    return w, op32, op64, m_true, d


def test_autograd_gradient_matches_central_differences(gm):
    import torch

    w, op32, op64, m_true, d = _mag128_problem(gm)
    m0 = torch.as_tensor(W.random_vector(w.model_shape, 2), device="cuda") * 0.01
    m = m0.float().clone().requires_grad_(True)
    loss = 0.5 * ((gm.gravmag_apply(m, op32) - d.float()) ** 2).sum()
    loss.backward()
    g = m.grad.double()

    def L(x):
        r = op64.forward(x.contiguous()) - d
        return 0.5 * float((r * r).sum())

    rng = np.random.default_rng(2)
    m0d = m.detach().double()
    worst = 0.0
    for _ in range(32):
        v = torch.as_tensor(rng.standard_normal(w.model_shape), device="cuda")
        h = 1e-3 * float(m0d.norm()) / float(v.norm())
        fd = (L(m0d + h * v) - L(m0d - h * v)) / (2 * h)
        ad = float((g * v).sum())
        worst = max(worst, abs(fd - ad) / max(abs(fd), 1e-300))
    assert worst < 1e-4, worst
    op32.close()
    op64.close()


def test_fp32_dot_product_test(gm):
    import torch

    w, op32, op64, _, _ = _mag128_problem(gm)
    x = torch.as_tensor(W.random_vector(w.model_shape, 3), dtype=torch.float32, device="cuda")
    y = torch.as_tensor(W.random_vector(w.data_shape, 4), dtype=torch.float32, device="cuda")
    a = float((op32.forward(x).double() * y.double()).sum())
    b = float((x.double() * op32.transpose(y).double()).sum())
    assert abs(a - b) / (float(op32.forward(x).double().norm()) * float(y.double().norm())) < 1e-6
    op32.close()
    op64.close()


def test_autograd_double_backward_free_path_and_grad_of_sum(gm):
    """d/dm SUM(G m * w) = G^T w through the Function, for both precisions."""
    import torch

    w = W.WORKLOADS["mag64"]
    for prec in (gm.F64, gm.F32):
        op = gm.Operator.from_workload(w, precision=prec)
        m = torch.as_tensor(W.model("mag64"), dtype=op.dtype, device="cuda").requires_grad_(True)
        wt = torch.as_tensor(W.data("mag64"), dtype=op.dtype, device="cuda")
        (gm.gravmag_apply(m, op) * wt).sum().backward()
        ref = op.transpose(wt)
        assert torch.equal(m.grad, ref)
        op.close()


def _cpu_tikhonov(G, d, alpha):
    n = G.shape[1]
    return np.linalg.solve(G.T @ G + alpha * alpha * np.eye(n), G.T @ d)


@pytest.mark.parametrize("kind", [W.GRAVITY, W.MAGNETIC])
@pytest.mark.parametrize("prec", ["F64", "DF64"])
def test_cgls_converges_to_tikhonov_solution(gm, kind, prec):
    """200 CGLS iterations reach the exact regularised solution.  alpha = 0.3 ||G|| keeps the
    condition number of G^T G + alpha^2 I near 12, so CG's error bound (((sqrt(k)-1)/(sqrt(k)+1))^i)
    is far below rounding after 200 iterations."""
    import torch

    geom = O.Geometry.uniform(4, 3, 2, 20.0, 25.0, 15.0, px=1, py=1, kind=kind, incl_deg=50.0, decl_deg=8.0)
    G = O.dense(geom)
    d = W.random_vector((3, 4), 9)
    alpha = 0.3 * float(np.linalg.norm(G, 2))
    x_ref = _cpu_tikhonov(G, d.ravel(), alpha)
    op = gm.Operator(4, 3, 2, 20.0, 25.0, 15.0, px=1, py=1, kind=kind, incl_deg=50.0, decl_deg=8.0,
                     precision=getattr(gm, prec))
    dt = torch.as_tensor(d, device="cuda")
    x, res = op.cgls(dt, alpha, 200)
    assert rel_err(x.cpu().numpy(), x_ref) < 1e-9
    assert res[-1] == pytest.approx(np.linalg.norm(G @ x_ref - d.ravel()), rel=1e-9)
    assert res[0] == pytest.approx(np.linalg.norm(d), rel=1e-12)
    # warm start from the solution stays there
    x2, res2 = op.cgls(dt, alpha, 3, x0=x)
    assert rel_err(x2.cpu().numpy(), x_ref) < 1e-9
    op.close()


def test_cgls_mag128_inversion(gm):
    """50 iterations of Tikhonov CGLS (alpha = 1e-2) on 1 % noisy data of the block model."""
    import torch

    w, op32, op64, m_true, d = _mag128_problem(gm)
    op32.forward(d.new_zeros(op32.model_shape, dtype=torch.float32))
    n_fwd = op32.last_launch_count()
    op32.transpose(d.float())
    n_tr = op32.last_launch_count()
    x, res = op32.cgls(d.float(), 1e-2, 50)
    assert np.all(np.isfinite(res))
    assert res[-1] < 0.2 * res[0]
    assert np.all(np.diff(res) <= 1e-3 * res[0])  # data misfit (essentially) non-increasing
    # the recursively updated FP32 residual drifts from the true one by O(iters * eps32 * ||d||)
    r = float((op64.forward(x.double()) - d).norm())
    assert abs(r - res[-1]) < 1e-4 * res[0], (r, res[-1], res[0])
    # start-up: G x0, G^T r and 2 vector kernels; per iteration: G p, G^T r and 4 vector kernels
    # (the reductions finish their scalar step in the last block to arrive)
    assert op32.last_launch_count() == n_fwd + n_tr + 2 + 50 * (n_fwd + n_tr + 4)
    op32.close()
    op64.close()
