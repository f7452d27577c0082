"""Learned warm start for the Tikhonov CGLS inversion of gravity data.

A convolutional network (2-D encoder, 3-D decoder; the architecture and its
C ABI are in include/gm_warmstart.h) maps a data grid d[S][S] to a density
model m[16][S][S].  It is trained on pairs (m, G m + 1% noise) whose data come
from this library's FP32 forward product, and its prediction x0 = net(d)
starts gm_cgls.  CGLS from x0 = 0 stays the fallback and the yardstick: the
comparison reports the data misfit plain CGLS reaches and the iterations and
G / G^T applies the warm-started CGLS needs to reach it.

The paper has no network; it names the inversion these products serve as the
use of its fast operators (Sec. 1, Sec. 6).  Everything numeric here runs in
libgravmag.so: the network's forward, backward and Adam kernels, the forward
products that make the training data, and CGLS.  This module marshals
arguments, draws the seeded synthetic models and keeps the training loop.
"""
from __future__ import annotations

import concurrent.futures
import ctypes
import math
import threading

import numpy as np

from . import gravmag as G
from . import workloads as W

DEPTH = 16
_sig_lock = threading.Lock()
_sig_done = False


def _lib():
    global _sig_done
    lib = G.load()
    with _sig_lock:
        if not _sig_done:
            vp, ci, cf, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_int64
            sig = {
                "gm_net_create": (vp, [ci, ci, ci, ctypes.c_ulonglong]),
                "gm_net_destroy": (ci, [vp]),
                "gm_net_num_params": (i64, [vp]),
                "gm_net_set_scales": (ci, [vp, cf, cf]),
                "gm_net_forward": (ci, [vp, vp, vp, ci, vp]),
                "gm_net_train_step": (ci, [vp, vp, vp, ci, vp, ci, cf, ctypes.POINTER(cf), vp]),
                "gm_net_get_params": (ci, [vp, vp, i64, ci]),
                "gm_net_set_params": (ci, [vp, vp, i64, ci]),
                "gm_net_get_step": (ci, [vp, ctypes.POINTER(i64)]),
                "gm_net_set_step": (ci, [vp, i64]),
                "gm_net_last_launch_count": (ci, [vp]),
                "gm_net_set_data_term": (ci, [vp, vp, cf]),
                "gm_net_last_losses": (ci, [vp, ctypes.POINTER(cf), ctypes.POINTER(cf)]),
                "gm_conv3d": (ci, [ci, ci, ci, ci, ci, ci, ci, ci, ci, vp, vp, vp, vp, vp, vp, vp]),
                "gm_net_last_error": (ctypes.c_char_p, []),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _sig_done = True
    return lib


def _check(status):
    if status != G.GM_OK:
        raise G.GravMagError(status, _lib().gm_net_last_error().decode(errors="replace"))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _device_f32(t, shape, name):
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return _ptr(t)


class WarmStartNet:
    """The network behind gm_net_*: FP32 master weights, BF16 convolution weights, Adam state."""

    PARAM_WHICH = {"weights": 0, "grad": 1, "adam_m": 2, "adam_v": 3}

    def __init__(self, grid: int = 64, max_batch: int = 32, seed: int = 0):
        h = _lib().gm_net_create(int(grid), DEPTH, int(max_batch), ctypes.c_ulonglong(seed))
        if not h:
            raise G.GravMagError(G.GM_EINVAL, _lib().gm_net_last_error().decode(errors="replace"))
        self._h = ctypes.c_void_p(h)
        self.grid, self.max_batch = int(grid), int(max_batch)
        self.in_scale, self.out_scale = 1.0, 1.0

    @property
    def num_params(self) -> int:
        return int(_lib().gm_net_num_params(self._h))

    def set_scales(self, in_scale: float, out_scale: float) -> None:
        _check(_lib().gm_net_set_scales(self._h, float(in_scale), float(out_scale)))
        self.in_scale, self.out_scale = float(in_scale), float(out_scale)

    def forward(self, d, out=None, stream=None):
        """net(d) for d of shape (B, S, S) -> (B, 16, S, S), float32 CUDA tensors."""
        import torch

        if d.dim() == 2:
            return self.forward(d.unsqueeze(0), None if out is None else out.unsqueeze(0), stream)[0]
        b = int(d.shape[0])
        if out is None:
            out = torch.empty((b, DEPTH, self.grid, self.grid), dtype=torch.float32, device=d.device)
        _check(_lib().gm_net_forward(self._h, _device_f32(d, (b, self.grid, self.grid), "d"),
                                     _device_f32(out, (b, DEPTH, self.grid, self.grid), "out"), b,
                                     G._stream_ptr(stream)))
        return out

    def train_step(self, d, m, lr: float, index=None, stream=None, want_loss: bool = True):
        """Loss and gradient on one batch, then an Adam step when lr > 0; returns the loss.

        Without `index`, d (B, S, S) and m (B, 16, S, S) are the batch; with it (a contiguous
        int32 CUDA tensor of B example numbers), d and m are whole example sets and the batch is
        gathered from them inside the network's input kernels."""
        import torch

        if index is None:
            b = int(d.shape[0])
            ip = None
        else:
            if not (index.is_cuda and index.dtype == torch.int32 and index.is_contiguous() and index.dim() == 1):
                raise TypeError("index must be a contiguous 1-D int32 CUDA tensor")
            b = int(index.shape[0])
            ip = _ptr(index)
        count = int(d.shape[0])
        if int(m.shape[0]) != count:
            raise ValueError("d and m hold different numbers of examples")
        loss = ctypes.c_float(0.0)
        _check(_lib().gm_net_train_step(self._h, _device_f32(d, (count, self.grid, self.grid), "d"),
                                        _device_f32(m, (count, DEPTH, self.grid, self.grid), "m"), count, ip, b,
                                        float(lr), ctypes.byref(loss) if want_loss else None,
                                        G._stream_ptr(stream)))
        return float(loss.value) if want_loss else None

    def set_data_term(self, op, lam: float) -> None:
        """Add lam * mean((in_scale (G net(d) - d))^2) to the training loss, with G = op (an FP32
        operator on the network's grid, S x S stations, no padding, 16 layers); lam = 0 removes it."""
        _check(_lib().gm_net_set_data_term(self._h, op.handle if op is not None else None, float(lam)))
        self._op = op if lam > 0 else None  # keep the operator alive while the network uses it

    def last_losses(self):
        """(model term, data term) of the last train step that read its loss back."""
        a, b = ctypes.c_float(0), ctypes.c_float(0)
        _check(_lib().gm_net_last_losses(self._h, ctypes.byref(a), ctypes.byref(b)))
        return float(a.value), float(b.value)

    def get_params(self, which: str = "weights") -> np.ndarray:
        out = np.empty(self.num_params, dtype=np.float32)
        _check(_lib().gm_net_get_params(self._h, ctypes.c_void_p(out.ctypes.data), out.size,
                                        self.PARAM_WHICH[which]))
        return out

    def set_params(self, values, which: str = "weights") -> None:
        a = np.ascontiguousarray(np.asarray(values, dtype=np.float32))
        _check(_lib().gm_net_set_params(self._h, ctypes.c_void_p(a.ctypes.data), a.size, self.PARAM_WHICH[which]))

    @property
    def step(self) -> int:
        s = ctypes.c_int64(0)
        _check(_lib().gm_net_get_step(self._h, ctypes.byref(s)))
        return int(s.value)

    def last_launch_count(self) -> int:
        return int(_lib().gm_net_last_launch_count(self._h))

    def save(self, path: str) -> None:
        """Checkpoint: weights, Adam moments, step count and scales (numpy .npz)."""
        np.savez(path, weights=self.get_params("weights"), adam_m=self.get_params("adam_m"),
                 adam_v=self.get_params("adam_v"), step=self.step, grid=self.grid,
                 scales=np.array([self.in_scale, self.out_scale]))

    def load(self, path: str) -> None:
        """Resume from save(): the next train_step continues the same Adam trajectory."""
        z = np.load(path)
        if int(z["grid"]) != self.grid:
            raise ValueError(f"checkpoint grid {int(z['grid'])} != {self.grid}")
        self.set_params(z["weights"], "weights")
        self.set_params(z["adam_m"], "adam_m")
        self.set_params(z["adam_v"], "adam_v")
        _check(_lib().gm_net_set_step(self._h, int(z["step"])))
        self.set_scales(*[float(v) for v in z["scales"]])

    def close(self) -> None:
        if getattr(self, "_h", None):
            _lib().gm_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def conv3d(mode: int, w, x=None, g=None, b=None, stride: int = 1, out=None, bias_grad=None, stream=None):
    """One convolution through the network's tensor-core kernels (see gm_conv3d): mode 0 forward
    (x -> out), 1 data gradient (g -> out), 2 weight gradient (x, g -> out [, bias_grad]).
    w is (CO, CI, KD, 3, 3); x (N, CI, D, H, W); g (N, CO, D, OH, OW); float32 CUDA tensors."""
    import torch

    CO, CI, KD = int(w.shape[0]), int(w.shape[1]), int(w.shape[2])
    if mode == 1:
        N, _, D, OH, OW = (int(v) for v in g.shape)
        if out is None:
            raise ValueError("mode 1 needs `out` (its input size is not implied by g)")
        IH, IW = int(out.shape[3]), int(out.shape[4])
    else:
        N, _, D, IH, IW = (int(v) for v in x.shape)
    OH, OW = (IH - 1) // stride + 1, (IW - 1) // stride + 1
    if out is None:
        shape = (N, CO, D, OH, OW) if mode == 0 else (CO, CI, KD, 3, 3)
        out = torch.empty(shape, dtype=torch.float32, device=w.device)
    chk = {"w": (w, (CO, CI, KD, 3, 3)), "out": (out, (N, CO, D, OH, OW) if mode == 0 else
                                                  (N, CI, D, IH, IW) if mode == 1 else (CO, CI, KD, 3, 3))}
    if mode != 1:
        chk["x"] = (x, (N, CI, D, IH, IW))
    if mode != 0:
        chk["g"] = (g, (N, CO, D, OH, OW))
    if b is not None:
        chk["b"] = (b, (CO,))
    if bias_grad is not None:
        chk["bias_grad"] = (bias_grad, (CO,))
    ptr = {k: _device_f32(t, shp, k) for k, (t, shp) in chk.items()}
    _check(_lib().gm_conv3d(int(mode), N, CI, CO, D, IH, IW, KD, int(stride), ptr.get("x"), ptr.get("g"), ptr["w"],
                            ptr.get("b"), ptr["out"], ptr.get("bias_grad"), G._stream_ptr(stream)))
    return out


# ------------------------------------------------------------------------------------------
# training data: seeded models, their FP32 forward data plus noise

def training_models(count: int, seed: int, shape=(DEPTH, 64, 64), threads: int = 0) -> np.ndarray:
    """`count` models (float32, (count, 16, S, S)); model i is drawn from rng (seed, i, 0x57) so the
    set does not depend on the thread count."""
    out = np.empty((count,) + tuple(shape), dtype=np.float32)

    def one(i):
        out[i] = W.training_model(np.random.default_rng((seed, i, 0x57)), shape)

    threads = threads or min(16, max(1, (__import__("os").cpu_count() or 1)))
    with concurrent.futures.ThreadPoolExecutor(threads) as ex:
        list(ex.map(one, range(count)))
    return out


def make_data(op: "G.Operator", models, noise_level: float, seed: int):
    """d_i = G m_i (this library's FP32 forward) + Gaussian noise of standard deviation
    noise_level * rms(G m_i), noise drawn from rng (seed, i, 0x4E).  `models` is a float32 CUDA
    tensor (count, 16, S, S); returns (clean, noisy) float32 CUDA tensors (count, S, S) and the
    noisy set on the host (float64)."""
    import torch

    count = int(models.shape[0])
    clean = torch.empty((count,) + tuple(op.data_shape), dtype=torch.float32, device=models.device)
    for i in range(count):
        op.forward(models[i], out=clean[i])
    host = clean.cpu().numpy().astype(np.float64)
    noisy = np.empty_like(host)
    for i in range(count):
        rms = float(np.sqrt(np.mean(host[i] ** 2)))
        noisy[i] = host[i] + np.random.default_rng((seed, i, 0x4E)).standard_normal(host[i].shape) * (
            noise_level * rms)
    return clean, torch.as_tensor(noisy.astype(np.float32)).to(models.device), noisy


def fit_scales(models: np.ndarray, data: np.ndarray):
    """in_scale = 1 / rms(data), out_scale = rms(models), over the training set."""
    return 1.0 / float(np.sqrt(np.mean(np.square(data, dtype=np.float64)))), \
        float(np.sqrt(np.mean(np.square(models, dtype=np.float64))))


def train(net: WarmStartNet, models, data, steps: int, batch: int, lr: float = 1e-3, seed: int = 0,
          lr_final: float | None = None, log_every: int = 0, record_every_loss: bool = True, stream=None):
    """Adam on minibatches drawn without replacement from a seeded permutation per epoch (the
    gather runs inside the network's input kernels); the learning rate decays by a cosine from
    lr to lr_final (default lr / 20).  Returns the loss of every step (None where not read back:
    reading it synchronises)."""
    import torch

    count = int(models.shape[0])
    if batch > net.max_batch or batch > count:
        raise ValueError("batch larger than the network's max_batch or the training set")
    lr_final = lr / 20 if lr_final is None else lr_final
    losses = []
    perm, pos, epoch = None, count, 0
    for k in range(steps):
        if pos + batch > count:
            perm = torch.as_tensor(np.random.default_rng((seed, epoch, 0xE9)).permutation(count).astype(np.int32),
                                   device=data.device)
            pos, epoch = 0, epoch + 1
        rate = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * k / max(1, steps - 1)))
        want = bool(log_every) or k == steps - 1 or record_every_loss
        losses.append(net.train_step(data, models, rate, index=perm[pos:pos + batch], stream=stream,
                                     want_loss=want))
        pos += batch
        if log_every and (k % log_every == 0 or k == steps - 1):
            print(f"step {k:6d}  lr {rate:.2e}  loss {losses[-1]:.4e}", flush=True)
    return losses


# ------------------------------------------------------------------------------------------
# the comparison: plain CGLS from zero against CGLS from the network's prediction

def iterations_to_reach(residuals, target) -> int | None:
    """First k with ||G x_k - d|| <= target, from a CGLS residual history (k = 0 is x0)."""
    for k, r in enumerate(residuals):
        if r <= target:
            return k
    return None


def cgls_applies(iterations: int, warm: bool) -> int:
    """G / G^T applies CGLS makes for k iterations: r0 = d - G x0 (skipped for x0 = 0),
    s0 = G^T r0, and one G and one G^T per iteration."""
    return (1 if warm else 0) + 1 + 2 * iterations


def compare(op: "G.Operator", net: WarmStartNet, d, m_true=None, alpha: float = 1e-2, plain_iters: int = 50,
            max_warm_iters: int | None = None, discrepancy: float | None = None):
    """Plain CGLS from zero against CGLS from x0 = net(d) on the same Tikhonov system.

    Plain CGLS stops at the first iteration whose misfit ||G x_k - d|| is at most `discrepancy`
    (the discrepancy principle; without it, after `plain_iters` iterations); its misfit there is
    the target.  The warm start stops at the first iteration that reaches the target.  Returns
    a dict: the target, the iterations and G / G^T applies each run needs, the misfit of x0,
    and (with m_true) the relative model errors of x0 and of both runs at their stopping
    iterations."""
    import torch

    max_warm_iters = plain_iters if max_warm_iters is None else max_warm_iters
    _, res_plain = op.cgls(d, alpha, plain_iters)
    k_plain = plain_iters
    if discrepancy is not None:
        k = iterations_to_reach(res_plain, discrepancy)
        k_plain = plain_iters if k is None else k
    target = float(res_plain[k_plain])
    x0 = net.forward(d.reshape(1, *d.shape))[0]
    _, res_warm = op.cgls(d, alpha, max_warm_iters, x0=x0)
    k_warm = iterations_to_reach(res_warm, target)
    out = {
        "alpha": alpha,
        "target_misfit": target,
        "plain_iterations": k_plain,
        "plain_applies": cgls_applies(k_plain, False),
        "warm_iterations": k_warm,
        "warm_applies": None if k_warm is None else cgls_applies(k_warm, True),
        "x0_misfit": float(res_warm[0]),
        "data_norm": float(d.double().norm()),
        "plain_residuals": [float(r) for r in res_plain],
        "warm_residuals": [float(r) for r in res_warm],
    }
    if m_true is not None:
        mt = m_true.double()
        nrm = float(mt.norm())
        x_plain, _ = op.cgls(d, alpha, k_plain)  # CGLS is deterministic: the same iterates again
        out["x0_model_error"] = float((x0.double() - mt).norm()) / nrm
        out["plain_model_error"] = float((x_plain.double() - mt).norm()) / nrm
        if k_warm is not None:
            x_warm, _ = op.cgls(d, alpha, k_warm, x0=x0)
            out["warm_model_error"] = float((x_warm.double() - mt).norm()) / nrm
    torch.cuda.synchronize()
    return out


def report(count: int = 20000, steps: int = 6000, batch: int = 32, lr: float = 1e-3, lam: float = 0.0,
           tests: int = 32, alpha: float = 1e-2, noise: float = 0.01, seed: int = 0, max_iters: int = 60,
           save: str | None = None, log_every: int = 500):
    """Train on `count` seeded pairs of the 64 x 64 x 16 gravity grid and compare warm-started with
    plain CGLS on `tests` held-out pairs (discrepancy principle with the known noise norm)."""
    import time

    import torch

    w = W.WORKLOADS["grav64"]
    op = G.Operator.from_workload(w, precision=G.F32)
    t0 = time.perf_counter()
    models_np = training_models(count + tests, seed=seed * 1000 + 1)
    models = torch.as_tensor(models_np).cuda()
    clean, noisy, noisy_np = make_data(op, models, noise, seed=seed * 1000 + 2)
    gen_s = time.perf_counter() - t0
    tr_m, tr_d = models[:count].contiguous(), noisy[:count].contiguous()
    net = WarmStartNet(grid=w.sx, max_batch=batch, seed=seed * 1000 + 3)
    net.set_scales(*fit_scales(models_np[:count], noisy_np[:count]))
    if lam > 0:
        net.set_data_term(op, lam)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = train(net, tr_m, tr_d, steps, batch, lr=lr, seed=seed, log_every=log_every, record_every_loss=False)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    if save:
        net.save(save)
    # inference and apply timing (CUDA events, after warm-up)
    d1 = noisy[count:count + 1].contiguous()
    for _ in range(3):
        net.forward(d1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        net.forward(d1)
    e1.record()
    torch.cuda.synchronize()
    infer_ms = e0.elapsed_time(e1) / 20
    m1 = models[count].contiguous()
    e0.record()
    for _ in range(20):
        op.forward(m1)
        op.transpose(d1[0])
    e1.record()
    torch.cuda.synchronize()
    apply_ms = e0.elapsed_time(e1) / 40
    rows = []
    for i in range(count, count + tests):
        e = float((noisy[i].double() - clean[i].double()).norm())
        r = compare(op, net, noisy[i].contiguous(), models[i], alpha=alpha, plain_iters=max_iters,
                    max_warm_iters=max_iters, discrepancy=e)
        r.pop("plain_residuals")
        r.pop("warm_residuals")
        r["noise_norm"] = e
        rows.append(r)
    reached = [r for r in rows if r["warm_applies"] is not None]

    def mean(key, rs=rows):
        vals = [r[key] for r in rs if r.get(key) is not None]
        return float(np.mean(vals)) if vals else None

    summary = {
        "workload": "grav64: gravity 64x64 stations, 16 layers of 25 m cells, no padding",
        "train_pairs": count, "steps": steps, "batch": batch, "lr": lr, "data_term_lambda": lam,
        "noise": noise, "alpha": alpha, "tests": tests, "params": net.num_params,
        "final_loss": losses[-1], "last_losses": net.last_losses(),
        "generate_s": gen_s, "train_s": train_s, "train_step_ms": 1e3 * train_s / max(1, steps),
        "net_forward_ms": infer_ms, "apply_ms": apply_ms,
        "reached_target": len(reached),
        "mean_plain_applies": mean("plain_applies"), "mean_warm_applies": mean("warm_applies", reached),
        "mean_plain_applies_same_tests": mean("plain_applies", reached),
        "fewer_applies": sum(1 for r in reached if r["warm_applies"] < r["plain_applies"]),
        "more_applies": sum(1 for r in reached if r["warm_applies"] > r["plain_applies"]),
        "mean_x0_misfit_rel": float(np.mean([r["x0_misfit"] / r["data_norm"] for r in rows])),
        "mean_noise_rel": float(np.mean([r["noise_norm"] / r["data_norm"] for r in rows])),
        "mean_x0_model_error": mean("x0_model_error"), "mean_plain_model_error": mean("plain_model_error"),
        "mean_warm_model_error": mean("warm_model_error"),
        "per_test": rows,
    }
    net.close()
    op.close()
    return summary


def _main(argv=None):
    import argparse
    import json

    ap = argparse.ArgumentParser(description="train the warm-start network and compare with plain CGLS")
    ap.add_argument("--count", type=int, default=20000)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lam", type=float, default=0.0)
    ap.add_argument("--tests", type=int, default=32)
    ap.add_argument("--alpha", type=float, default=1e-2)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--save", default=None)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    s = report(a.count, a.steps, a.batch, a.lr, a.lam, a.tests, a.alpha, seed=a.seed, save=a.save)
    brief = {k: v for k, v in s.items() if k != "per_test"}
    print(json.dumps(brief), flush=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(s, f, indent=1)


if __name__ == "__main__":
    _main()
