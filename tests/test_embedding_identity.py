"""The BCCB embedding of Sec. 3 checked on the CPU (no GPU, no product code).

These tests restate, with numpy's FFT and oracle entries, the identity the
CUDA path is built on (Eq. GrviaT with the padded W of Eqs. Wpadded and
WTpadded): d = window(IFFT2(SUM_r FFT2(T_r) .* FFT2(W_r))), and the transpose
with conj(FFT2(T_r)), for any FFT length N' >= s + n - 1 per axis.  They pin the
generator index map (u = i - p stored at u mod N', v = j - q at v mod N')
against the dense oracle, so that a GPU mismatch later is a kernel bug, not a
misreading of the paper.
"""
import numpy as np
import pytest

import oracle as O
from paper_1912_06976_gb300 import workloads as W
from tests.conftest import rel_err


def _generator(geom, Nx, Ny):
    """t_r(u, v) = G[(j,i), (r,q,p)] with u = i - p, v = j - q, stored at (v mod Ny, u mod Nx)."""
    T = np.zeros((geom.nz, Ny, Nx))
    for r in range(geom.nz):
        for v in range(-(geom.ny - 1), geom.sy):
            j = max(v, 0)
            q = j - v
            for u in range(-(geom.nx - 1), geom.sx):
                i = max(u, 0)
                p = i - u
                T[r, v % Ny, u % Nx] = O.entry(geom, i, j, p, q, r)
    return T


def _fft_forward(geom, T, m):
    nz, Ny, Nx = T.shape
    acc = np.zeros((Ny, Nx), dtype=complex)
    for r in range(nz):
        Wr = np.zeros((Ny, Nx))
        Wr[:geom.ny, :geom.nx] = m[r]
        acc += np.fft.fft2(T[r]) * np.fft.fft2(Wr)
    return np.real(np.fft.ifft2(acc))[:geom.sy, :geom.sx]


def _fft_transpose(geom, T, d):
    nz, Ny, Nx = T.shape
    V = np.zeros((Ny, Nx))
    V[:geom.sy, :geom.sx] = d
    Vh = np.fft.fft2(V)
    return np.stack([np.real(np.fft.ifft2(np.conj(np.fft.fft2(T[r])) * Vh))[:geom.ny, :geom.nx]
                     for r in range(nz)])


def _geom(w):
    return O.Geometry(w.sx, w.sy, w.nz, w.dx, w.dy, w.zplanes, w.pxl, w.pxr, w.pyl, w.pyr,
                      w.kind, w.incl_deg, w.decl_deg, w.F_nT)


@pytest.mark.parametrize("seed,kind", [(1, W.GRAVITY), (2, W.MAGNETIC), (3, W.MAGNETIC), (4, W.GRAVITY)])
@pytest.mark.parametrize("extra", [0, 5])
def test_circulant_embedding_matches_dense(seed, kind, extra):
    w = W.random_shape_workload(seed, kind)
    geom = _geom(w)
    Nx, Ny = w.sx + w.nx - 1 + extra, w.sy + w.ny - 1 + extra
    T = _generator(geom, Nx, Ny)
    rng = np.random.default_rng(seed)
    m = rng.standard_normal(w.model_shape)
    d = rng.standard_normal(w.data_shape)
    assert rel_err(_fft_forward(geom, T, m), O.forward(geom, m)) < 1e-13
    assert rel_err(_fft_transpose(geom, T, d), O.transpose(geom, d)) < 1e-13


def test_sec3_three_by_three_circulant_example():
    """Sec. 3: the 3x3 Toeplitz with first row (g1, g2, g3) and first column (g1, gam2, gam3)
    sits in the top-left corner of the 5x5 circulant whose first column is
    (g1, gam2, gam3, g3, g2) -- the paper's minimal extension without the extra 0."""
    geom = O.Geometry(3, 1, 1, 20.0, 20.0, (0.0, 20.0), 0, 0, 0, 0, O.MAGNETIC, 50.0, 8.0)
    G = O.dense(geom)
    g1, g2, g3 = G[0, 0], G[0, 1], G[0, 2]
    gam2, gam3 = G[1, 0], G[2, 0]
    T = _generator(geom, 5, 1)[0, 0]
    # the circulant C[a, b] = c[(a - b) mod 5] acts as d = C m: its first column is t(u), u = a - 0
    np.testing.assert_array_equal(T, [g1, gam2, gam3, g3, g2])
    C = np.array([[T[(a - b) % 5] for b in range(5)] for a in range(5)])
    np.testing.assert_array_equal(C[:3, :3], G)
