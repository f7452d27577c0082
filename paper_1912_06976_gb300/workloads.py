"""Seeded synthetic workloads shaped like the paper's problems.

This module holds no part of the operator's arithmetic: it only describes the
five geometries the library is exercised on and draws seeded model and data
vectors for them with ``numpy.random.default_rng`` (PCG64, identical on x86-64
and aarch64).  Tests feed the same arrays to the CPU oracle and to the CUDA
path.

Layouts follow Sec. 2 of Hogue, Renaut & Vatankhah (arXiv 1912.06976), Eqs.
Gslice and htilde: a model is ``m[r, q, p]`` (depth, y, x; x fastest) over the
padded cell grid, data are ``d[j, i]`` (x fastest) over the stations.

The paper itself draws only random vectors (Sec. 5); the structured models
below (blocks, dipping slabs, Gaussian random fields) stand in for the kind of
density / susceptibility volumes the method is meant for.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GRAVITY = 0
MAGNETIC = 1


@dataclasses.dataclass(frozen=True)
class Workload:
    """One geometry: sx, sy stations, nz layers, cell sizes (m), pads per side."""

    name: str
    kind: int
    sx: int
    sy: int
    nz: int
    dx: float
    dy: float
    dz: float
    px: int
    py: int
    incl_deg: float = 90.0
    decl_deg: float = 0.0
    F_nT: float = 50000.0
    pxr_: int = -1  # right / far padding when it differs from px (Sec. 2.1.2 allows p_L != p_R)
    pyr_: int = -1

    @property
    def pxl(self) -> int:
        return self.px

    @property
    def pyl(self) -> int:
        return self.py

    @property
    def pxr(self) -> int:
        return self.px if self.pxr_ < 0 else self.pxr_

    @property
    def pyr(self) -> int:
        return self.py if self.pyr_ < 0 else self.pyr_

    @property
    def nx(self) -> int:
        return self.sx + self.pxl + self.pxr

    @property
    def ny(self) -> int:
        return self.sy + self.pyl + self.pyr

    @property
    def zplanes(self):
        return tuple(k * self.dz for k in range(self.nz + 1))

    @property
    def m(self) -> int:
        return self.sx * self.sy

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def model_shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def data_shape(self):
        return (self.sy, self.sx)


WORKLOADS = {
    # 16 x 16 stations over 8 layers of 50 m cubes, gravity, no padding.
    "grav16": Workload("grav16", GRAVITY, 16, 16, 8, 50.0, 50.0, 50.0, 0, 0),
    # 64 x 64 stations, 16 layers of 25 m cells, 3 pad cells per side, magnetic I=50 D=8.
    "mag64": Workload("mag64", MAGNETIC, 64, 64, 16, 25.0, 25.0, 25.0, 3, 3, 50.0, 8.0),
    # 300 x 250 stations, 60 layers of 20 m cells, 10 % padding per side (30 / 25 cells), gravity.
    "grav300": Workload("grav300", GRAVITY, 300, 250, 60, 20.0, 20.0, 20.0, 30, 25),
    # 128 x 128 stations, 32 layers of 25 m cells, no padding, magnetic I=60 D=0.
    "mag128": Workload("mag128", MAGNETIC, 128, 128, 32, 25.0, 25.0, 25.0, 0, 0, 60.0, 0.0),
    # 64 x 64 stations, 16 layers of 25 m cells, no padding, gravity (warm-start training grid).
    "grav64": Workload("grav64", GRAVITY, 64, 64, 16, 25.0, 25.0, 25.0, 0, 0),
}


def _set_block(m, x0, x1, y0, y1, z0, z1, value, add=False):
    if add:
        m[z0:z1, y0:y1, x0:x1] += value
    else:
        m[z0:z1, y0:y1, x0:x1] = value


def gaussian_random_field(rng, shape, corr_cells, sigma):
    """White noise filtered by exp(-k^2 l^2 / 2) in 3-D, scaled to standard deviation sigma."""
    w = rng.standard_normal(shape)
    ks = [np.fft.fftfreq(s) * 2.0 * math.pi for s in shape]
    kz, ky, kx = np.meshgrid(*ks, indexing="ij", sparse=True)
    filt = np.exp(-(kx * kx + ky * ky + kz * kz) * corr_cells * corr_cells / 2.0)
    f = np.real(np.fft.ifftn(np.fft.fftn(w) * filt))
    f -= f.mean()
    return f * (sigma / max(f.std(), 1e-300))


def random_blocks(rng, shape, count, side_x, side_y, side_z, low, high, signed=False):
    """Sum of `count` rectangular bodies with integer sides drawn from the given ranges."""
    nz, ny, nx = shape
    m = np.zeros(shape)
    for _ in range(count):
        sx = int(rng.integers(side_x[0], side_x[1] + 1))
        sy = int(rng.integers(side_y[0], side_y[1] + 1))
        sz = int(rng.integers(side_z[0], side_z[1] + 1))
        sx, sy, sz = min(sx, nx), min(sy, ny), min(sz, nz)
        x0 = int(rng.integers(0, nx - sx + 1))
        y0 = int(rng.integers(0, ny - sy + 1))
        z0 = int(rng.integers(0, nz - sz + 1))
        v = float(rng.uniform(low, high))
        if signed and rng.random() < 0.5:
            v = -v
        m[z0:z0 + sz, y0:y0 + sy, x0:x0 + sx] += v
    return m


def model(name: str, seed: int = 0) -> np.ndarray:
    """The seeded model vector of a named workload, shape (nz, ny, nx), float64."""
    w = WORKLOADS[name]
    rng = np.random.default_rng(seed)
    shape = w.model_shape
    if name == "grav16":
        m = rng.uniform(0.0, 0.1, shape)
        _set_block(m, 3, 7, 3, 7, 2, 4, 1.0)
        _set_block(m, 9, 13, 8, 12, 4, 6, 1.0)
        return m
    if name == "mag64":
        m = rng.uniform(0.0, 0.01, shape)
        nz, ny, nx = shape
        r = np.arange(nz)[:, None, None]
        q = np.arange(ny)[None, :, None]
        p = np.arange(nx)[None, None, :]
        for x0, dip, ztop in ((20, 30.0, 1), (35, 45.0, 2), (50, 60.0, 3)):
            cot = 1.0 / math.tan(math.radians(dip))
            inside = (np.abs(p - x0 - (r - ztop) * cot) < 1.5) & (r >= ztop) & (q >= 25) & (q < 45)
            m[inside] = 0.05
        return m
    if name == "grav300":
        m = gaussian_random_field(rng, shape, 8.0, 0.2)
        m += random_blocks(rng, shape, 20, (4, 40), (4, 40), (2, 15), 0.3, 1.0, signed=True)
        return m
    if name == "mag128":
        return random_blocks(rng, shape, 8, (8, 40), (8, 40), (3, 10), 0.01, 0.05)
    if name == "grav64":
        return training_model(rng, shape)
    raise KeyError(name)


def training_model(rng, shape) -> np.ndarray:
    """One warm-start training model: random blocks, or a Gaussian random field plus blocks."""
    if rng.random() < 0.5:
        return random_blocks(rng, shape, int(rng.integers(1, 6)), (4, 24), (4, 24), (2, 8), 0.1, 1.0)
    corr = float(rng.uniform(4.0, 12.0))
    m = gaussian_random_field(rng, shape, corr, 0.1)
    return m + random_blocks(rng, shape, int(rng.integers(1, 4)), (4, 24), (4, 24), (2, 8), 0.1, 1.0)


def data(name: str, seed: int = 0) -> np.ndarray:
    """A seeded data vector d ~ N(0, 1) for the transpose product, shape (sy, sx).

    The stream is seeded with (seed, 0xD), independent of the model stream."""
    w = WORKLOADS[name]
    rng = np.random.default_rng((seed, 0xD))
    return rng.standard_normal(w.data_shape)


def noise(d: np.ndarray, level: float, seed: int) -> np.ndarray:
    """Gaussian noise with standard deviation level * ||d||_2 / sqrt(len(d))."""
    rng = np.random.default_rng(seed)
    sig = level * float(np.linalg.norm(d)) / math.sqrt(d.size)
    return rng.standard_normal(d.shape) * sig


def random_shape_workload(seed: int, kind: int) -> Workload:
    """A small geometry with odd, unequal sizes and asymmetric padding for parity sweeps."""
    rng = np.random.default_rng((seed, 0x5A))
    sx, sy = int(rng.integers(1, 24)), int(rng.integers(1, 24))
    return Workload(f"rand{seed}", kind, sx, sy, int(rng.integers(1, 5)),
                    float(rng.uniform(5, 60)), float(rng.uniform(5, 60)), float(rng.uniform(5, 60)),
                    int(rng.integers(0, 5)), int(rng.integers(0, 5)),
                    float(rng.uniform(-90, 90)), float(rng.uniform(-180, 180)), 50000.0,
                    int(rng.integers(0, 5)), int(rng.integers(0, 5)))


def random_vector(shape, seed: int) -> np.ndarray:
    """A seeded N(0, 1) vector, e.g. the paper's random u and v of Sec. 5."""
    return np.random.default_rng((seed, 0x7E)).standard_normal(shape)
