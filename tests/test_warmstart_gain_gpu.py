"""What the trained network gains over CGLS without it (plain CGLS is the yardstick).

A network trained on the GPU with the library's kernels (8,192 seeded pairs of the 64 x 64 x 16
gravity grid, data from the FP32 forward product + 1 % noise, 3,000 Adam steps of batch 32) starts
Tikhonov CGLS (alpha = 1e-2) on 16 held-out pairs.  Plain CGLS from zero stops by the discrepancy
principle (misfit <= the known noise norm); the warm start must reach that misfit with fewer
G / G^T applies on average, and its model at that misfit must be closer to the true model.
(The full-size run, 20,000 pairs and 6,000 steps, is `python -m paper_1912_06976_gb300.warmstart`.)
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_warm_start_reaches_the_plain_misfit_with_fewer_applies(gm):
    import torch

    from paper_1912_06976_gb300 import warmstart as WS
    from paper_1912_06976_gb300 import workloads as W

    count, tests = 8192, 16
    w = W.WORKLOADS["grav64"]
    op = gm.Operator.from_workload(w, precision=gm.F32)
    models_np = WS.training_models(count + tests, seed=21)
    models = torch.as_tensor(models_np).cuda()
    clean, noisy, noisy_np = WS.make_data(op, models, 0.01, seed=22)
    net = WS.WarmStartNet(grid=64, max_batch=32, seed=23)
    net.set_scales(*WS.fit_scales(models_np[:count], noisy_np[:count]))
    losses = WS.train(net, models[:count].contiguous(), noisy[:count].contiguous(), 3000, 32, lr=1e-3, seed=24,
                      record_every_loss=False)
    assert np.isfinite(losses[-1]) and losses[-1] < 0.6  # the normalised model loss starts near 1
    rows = []
    for i in range(count, count + tests):
        e = float((noisy[i].double() - clean[i].double()).norm())
        rows.append(WS.compare(op, net, noisy[i].contiguous(), models[i], alpha=1e-2, plain_iters=60,
                               max_warm_iters=60, discrepancy=e))
    assert all(r["warm_applies"] is not None for r in rows)  # every warm start reaches the target
    plain = np.mean([r["plain_applies"] for r in rows])
    warm = np.mean([r["warm_applies"] for r in rows])
    assert warm < plain, (warm, plain)
    err_plain = np.mean([r["plain_model_error"] for r in rows])
    err_warm = np.mean([r["warm_model_error"] for r in rows])
    assert err_warm < 0.85 * err_plain, (err_warm, err_plain)
    net.close()
    op.close()
