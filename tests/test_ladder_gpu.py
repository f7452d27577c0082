"""Every FFT length of the register-codelet ladder, in the row and the column direction, FP32,
FP64 and double-float (DF64): against the oracle at sampled stations and cells, and over the
whole vector against the generic kernels (selected with GM_GENERIC_FFT=1; DF64, which has no
generic kernels, against the FP64 codelet run).

A geometry with s stations and no padding has N = 2 s - 1; s = L / 2 makes the plan pick the
ladder length L.  The other direction is kept at 16 stations (length 32), with two layers and a
magnetic kernel every other case so that both spectra kinds run on every length."""
import numpy as np
import pytest

import oracle as O
from paper_1912_06976_gb300 import workloads as W
from tests.conftest import assert_close, rel_err

pytestmark = pytest.mark.gpu

X_LADDER = [32, 48, 64, 80, 96, 112, 128, 140, 160, 192, 224, 256, 288, 320, 384, 448, 512, 560, 576, 640, 672,
            768, 896, 1024]
Y_LADDER = [32, 48, 64, 80, 96, 112, 128, 140, 160, 192, 224, 256, 288, 320, 384, 448, 512, 560, 576, 640, 672, 768]
TOL = {1: 1e-12, 0: 1e-5, 2: 1e-12}


def _case(direction, L, i):
    s = L // 2
    sx, sy = (s, 16) if direction == "x" else (16, s)
    kind = W.MAGNETIC if i % 2 else W.GRAVITY
    return W.Workload(f"{direction}{L}", kind, sx, sy, 2, 20.0, 25.0, 15.0, 0, 0, 55.0, 20.0)


CASES = [("x", L, i) for i, L in enumerate(X_LADDER)] + [("y", L, i) for i, L in enumerate(Y_LADDER)]


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("direction,L,i", CASES, ids=[f"{d}{L}" for d, L, _ in CASES])
def test_ladder_length_vs_oracle_and_generic(gm, monkeypatch, direction, L, i, prec):
    import torch

    w = _case(direction, L, i)
    geom = O.Geometry(w.sx, w.sy, w.nz, w.dx, w.dy, w.zplanes, w.pxl, w.pxr, w.pyl, w.pyr, w.kind, w.incl_deg,
                      w.decl_deg, w.F_nT)
    m = W.random_vector(w.model_shape, 40 + i)
    d = W.random_vector(w.data_shape, 80 + i)
    dt = torch.float32 if prec == 0 else torch.float64

    def run(p=prec):
        op = gm.Operator.from_workload(w, precision=p)
        info = op.get_info()
        f = op.forward(torch.as_tensor(m, dtype=dt, device="cuda")).double().cpu().numpy()
        t = op.transpose(torch.as_tensor(d, dtype=dt, device="cuda")).double().cpu().numpy()
        op.close()
        return info, f, t

    info, f, t = run()
    assert (info.fft_nx if direction == "x" else info.fft_ny) == L
    rng = np.random.default_rng(i)
    st = np.sort(rng.choice(w.sx * w.sy, size=min(48, w.sx * w.sy), replace=False))
    ce = np.sort(rng.choice(w.nx * w.ny * w.nz, size=48, replace=False))
    assert_close(f.ravel()[st], O.forward(geom, m, stations=st), TOL[prec])
    assert_close(t.ravel()[ce], O.transpose(geom, d, cells=ce), TOL[prec])
    if prec == 2:
        _, fg, tg = run(1)
    else:
        monkeypatch.setenv("GM_GENERIC_FFT", "1")
        _, fg, tg = run()
        monkeypatch.delenv("GM_GENERIC_FFT")
    tol = 3e-6 if prec == 0 else 1e-13
    assert_close(f, fg, tol)
    assert_close(t, tg, tol)
