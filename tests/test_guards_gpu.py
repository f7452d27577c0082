"""Guard regions around every caller buffer of the C ABI.

Each buffer handed to an entry point is the middle of a larger allocation whose other elements hold
a canary bit pattern.  After the call nothing outside the buffer may have changed, and an input
buffer must be unchanged inside too.  This catches out-of-range writes and writes to inputs, which
the value comparisons against the oracle would not see.  Sizes are odd, one workload has a single
layer, and both kinds and all three precisions are covered.  Buffers start on 16-byte boundaries:
the kernels access caller buffers element by element, so nothing here depends on the alignment.
"""
import numpy as np
import pytest

from paper_1912_06976_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GUARD = 1024  # elements of canary on each side (a multiple of 4: 16-byte aligned views)
CANARY32 = 0x7FC0BEEF  # a quiet-NaN pattern no kernel writes
CANARY64 = 0x7FF8DEADBEEFCAFE

CASES = [
    ("grav16", 1), ("grav16", 0), ("grav16", 2),
    ("mag64", 1), ("mag64", 2),
    ("odd1", 1), ("odd1", 0),
    ("oddmag", 1),
]


def workload(name):
    if name == "odd1":  # one layer, odd station counts, asymmetric padding
        return W.Workload("odd1", W.GRAVITY, 13, 7, 1, 10.0, 12.0, 8.0, 1, 2, 90.0, 0.0, 50000.0, 2, 3)
    if name == "oddmag":
        return W.Workload("oddmag", W.MAGNETIC, 11, 17, 3, 20.0, 15.0, 10.0, 2, 1, 35.0, -20.0, 48000.0, 3, 1)
    return W.WORKLOADS[name]


class Guarded:
    """A buffer of n elements inside 2*GUARD canary elements (device or page-locked host)."""

    def __init__(self, torch, n, dtype, where, fill=None):
        self.torch, self.n, self.dtype = torch, n, dtype
        it = torch.int32 if dtype == torch.float32 else torch.int64
        canary = CANARY32 if dtype == torch.float32 else CANARY64
        raw = torch.full((GUARD + n + GUARD,), canary, dtype=it)
        raw = raw.cuda() if where == "cuda" else raw.pin_memory()
        self.raw = raw
        self.bits = raw.view(dtype)
        self.buf = self.bits[GUARD:GUARD + n]
        if fill is not None:
            self.buf.copy_(fill.reshape(-1).to(dtype))
        self.before = raw.clone()

    def check(self, what, unchanged_inside):
        self.torch.cuda.synchronize()
        now, was = self.raw.cpu(), self.before.cpu()
        assert self.torch.equal(now[:GUARD], was[:GUARD]), f"{what}: write before the buffer"
        assert self.torch.equal(now[GUARD + self.n:], was[GUARD + self.n:]), f"{what}: write past the buffer"
        if unchanged_inside:
            assert self.torch.equal(now[GUARD:GUARD + self.n], was[GUARD:GUARD + self.n]), f"{what}: input modified"


@pytest.mark.parametrize("name,prec", CASES)
def test_operator_entry_points_stay_inside_their_buffers(gm, name, prec):
    import torch

    w = workload(name)
    op = gm.Operator.from_workload(w, precision=prec)
    dt = op.dtype
    n, m = op.info.n_model, op.info.n_data
    rng = np.random.default_rng(7)
    mv = torch.as_tensor(rng.standard_normal(n))
    dv = torch.as_tensor(rng.standard_normal(m))
    for where in ("cuda", "host"):
        gin_m, gout_d = Guarded(torch, n, dt, where, mv), Guarded(torch, m, dt, where)
        gin_d, gout_m = Guarded(torch, m, dt, where, dv), Guarded(torch, n, dt, where)
        if where == "cuda":
            op.forward(gin_m.buf, out=gout_d.buf)
            op.transpose(gin_d.buf, out=gout_m.buf)
        else:
            op.forward_host(gin_m.buf, gout_d.buf)
            op.transpose_host(gin_d.buf, gout_m.buf)
        for g, what, inp in ((gin_m, "forward input", True), (gout_d, "forward output", False),
                             (gin_d, "transpose input", True), (gout_m, "transpose output", False)):
            g.check(f"{where} {what}", inp)
        if where == "host":  # the stream-ordered forms, two calls each so that they chain
            s = torch.cuda.Stream()
            for _ in range(2):
                op.forward_host_async(gin_m.buf, gout_d.buf, stream=s)
                op.transpose_host_async(gin_d.buf, gout_m.buf, stream=s)
            s.synchronize()
            for g, what, inp in ((gin_m, "forward input", True), (gout_d, "forward output", False),
                                 (gin_d, "transpose input", True), (gout_m, "transpose output", False)):
                g.check(f"async {what}", inp)
    # CGLS: d and x0 are inputs, x the output (the handle's scratch and the fixed array are the
    # library's own)
    gd = Guarded(torch, m, dt, "cuda", dv)
    gx0 = Guarded(torch, n, dt, "cuda", 0.1 * mv)
    for fn in (op.cgls, op.cgls_noalloc):
        gx = Guarded(torch, n, dt, "cuda")
        fn(gd.buf, 1e-2, 3, x0=gx0.buf, out=gx.buf)
        gd.check(f"{fn.__name__} data", True)
        gx0.check(f"{fn.__name__} start", True)
        gx.check(f"{fn.__name__} iterate", False)
    op.close()


def test_network_forward_stays_inside_its_buffers(gm):
    import torch

    from paper_1912_06976_gb300 import warmstart as WS

    net = WS.WarmStartNet(grid=64, max_batch=4, seed=3)
    b, S, D = 3, 64, WS.DEPTH
    rng = np.random.default_rng(11)
    gin = Guarded(torch, b * S * S, torch.float32, "cuda", torch.as_tensor(rng.standard_normal(b * S * S)))
    gout = Guarded(torch, b * D * S * S, torch.float32, "cuda")
    net.forward(gin.buf.view(b, S, S), out=gout.buf.view(b, D, S, S))
    gin.check("network input", True)
    gout.check("network output", False)
