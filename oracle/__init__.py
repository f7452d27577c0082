"""CPU oracle for the gravity / magnetic prism operator G (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline leg, never by the product package.  The
arithmetic lives in ``gm_oracle.c`` (IEEE binary128, dense G entry by entry from
the prism formulas of Sec. 4 of Hogue, Renaut & Vatankhah, arXiv 1912.06976);
this module only builds that file with gcc and marshals numpy arrays through
ctypes.

Layouts follow Sec. 2 (Eqs. Gslice, htilde): model ``m[r, q, p]`` (x fastest)
and data ``d[j, i]`` (x fastest), flattened in C order.

Parity status: every function here is pinned by tests/test_oracle_pins.py
(point-mass and dipole limits, Bouguer slab, Gauss-Legendre quadrature,
sub-prism additivity, Laplace, symmetries, the Toeplitz invariant and the
worked examples of Sec. 2.2); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgm_oracle.so")

GRAVITY = 0
MAGNETIC = 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gm_oracle.c into oracle/_build/libgm_oracle.so (gcc, OpenMP if available).

    The arithmetic is binary128: long double where that is the format (aarch64), else
    __float128 with libquadmath (x86-64); gcc fails on a machine with neither.
    """
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
    last = None
    for extra_pre, extra_post in ((["-fopenmp"], ["-lquadmath"]), (["-fopenmp"], []), ([], ["-lquadmath"]), ([], [])):
        try:
            subprocess.run(base[:1] + extra_pre + base[1:] + extra_post, check=True, capture_output=True, text=True)
            break
        except subprocess.CalledProcessError as e:
            last = e
    else:
        raise RuntimeError(f"cannot build the oracle: {last.stderr if last else ''}")
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Geom(ctypes.Structure):
    _fields_ = [
        ("sx", ctypes.c_int), ("sy", ctypes.c_int), ("nz", ctypes.c_int),
        ("pxl", ctypes.c_int), ("pxr", ctypes.c_int), ("pyl", ctypes.c_int), ("pyr", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double),
        ("zplanes", ctypes.POINTER(ctypes.c_double)),
        ("kind", ctypes.c_int),
        ("incl_deg", ctypes.c_double), ("decl_deg", ctypes.c_double), ("F_nT", ctypes.c_double),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        gp = ctypes.POINTER(_Geom)
        lib.gmo_prism_grav.restype = ctypes.c_double
        lib.gmo_prism_grav.argtypes = [ctypes.c_double] * 6
        lib.gmo_prism_mag_terms.restype = None
        lib.gmo_prism_mag_terms.argtypes = [ctypes.c_double] * 6 + [dp]
        lib.gmo_mag_coeffs.restype = None
        lib.gmo_mag_coeffs.argtypes = [gp, dp]
        lib.gmo_entry.restype = ctypes.c_double
        lib.gmo_entry.argtypes = [gp] + [ctypes.c_int] * 5
        lib.gmo_rows.restype = None
        lib.gmo_rows.argtypes = [gp, i64p, ctypes.c_int64, dp]
        lib.gmo_entries.restype = None
        lib.gmo_entries.argtypes = [gp, i64p, i64p, ctypes.c_int64, dp]
        lib.gmo_forward.restype = None
        lib.gmo_forward.argtypes = [gp, dp, i64p, ctypes.c_int64, dp]
        lib.gmo_transpose.restype = None
        lib.gmo_transpose.argtypes = [gp, dp, i64p, ctypes.c_int64, dp]
        lib.gmo_threads.restype = ctypes.c_int
        lib.gmo_set_threads.argtypes = [ctypes.c_int]
        lib.gmo_mant_dig.restype = ctypes.c_int
        _lib = lib
        return lib


@dataclasses.dataclass(frozen=True)
class Geometry:
    """Station grid and prism volume (Sec. 2.1; notation table of App. A).

    sx, sy  stations in x and y (= unpadded cells per row / column)
    nz      depth layers
    pxl, pxr, pyl, pyr  padding cells left/right of the stations in x and y
    dx, dy  cell sizes (m); zplanes: nz+1 increasing layer boundaries (m),
            z down, zplanes[0] >= 0; the stations are at depth 0 (uniform
            layers: k*dz)
    kind    GRAVITY (m in g/cm^3, d in mGal) or MAGNETIC (m = susceptibility
            SI, d in nT; x North, y East)
    """

    sx: int
    sy: int
    nz: int
    dx: float
    dy: float
    zplanes: tuple
    pxl: int = 0
    pxr: int = 0
    pyl: int = 0
    pyr: int = 0
    kind: int = GRAVITY
    incl_deg: float = 90.0
    decl_deg: float = 0.0
    F_nT: float = 50000.0

    @staticmethod
    def uniform(sx, sy, nz, dx, dy, dz, px=0, py=0, kind=GRAVITY, incl_deg=90.0, decl_deg=0.0,
                F_nT=50000.0, pxr=None, pyr=None):
        return Geometry(sx, sy, nz, float(dx), float(dy), tuple(float(k * dz) for k in range(nz + 1)),
                        px, px if pxr is None else pxr, py, py if pyr is None else pyr,
                        kind, float(incl_deg), float(decl_deg), float(F_nT))

    @property
    def nx(self):
        return self.sx + self.pxl + self.pxr

    @property
    def ny(self):
        return self.sy + self.pyl + self.pyr

    @property
    def m(self):
        return self.sx * self.sy

    @property
    def n(self):
        return self.nx * self.ny * self.nz

    def _c(self):
        z = np.ascontiguousarray(self.zplanes, dtype=np.float64)
        assert z.shape == (self.nz + 1,)
        g = _Geom(self.sx, self.sy, self.nz, self.pxl, self.pxr, self.pyl, self.pyr,
                  self.dx, self.dy, z.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                  self.kind, self.incl_deg, self.decl_deg, self.F_nT)
        return g, z  # keep z alive alongside the struct


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def prism_grav(x1, x2, y1, y2, z1, z2) -> float:
    """Signed 8-corner gravity sum (without gamma) of one prism; station at the origin."""
    return _load().gmo_prism_grav(x1, x2, y1, y2, z1, z2)


def prism_mag_terms(x1, x2, y1, y2, z1, z2) -> np.ndarray:
    """{L_x, L_y, L_z, A_x, A_y, A_z} of one prism; station at the origin."""
    out = np.zeros(6)
    _load().gmo_prism_mag_terms(x1, x2, y1, y2, z1, z2, _dp(out))
    return out


def mag_coeffs(geom: Geometry) -> np.ndarray:
    """Coefficients of {L_x, L_y, L_z, A_x, A_y} in a magnetic entry (F/4pi included)."""
    out = np.zeros(5)
    g, _z = geom._c()
    _load().gmo_mag_coeffs(ctypes.byref(g), _dp(out))
    return out


def entry(geom: Geometry, i, j, p, q, r) -> float:
    g, _z = geom._c()
    return _load().gmo_entry(ctypes.byref(g), i, j, p, q, r)


def rows(geom: Geometry, stations) -> np.ndarray:
    """Dense rows G[k, :] for the listed stations k = j*sx + i."""
    st = np.ascontiguousarray(stations, dtype=np.int64)
    out = np.zeros((st.size, geom.n))
    g, _z = geom._c()
    _load().gmo_rows(ctypes.byref(g), _ip(st), st.size, _dp(out))
    return out


def entries(geom: Geometry, stations, cells) -> np.ndarray:
    """G[stations[t], cells[t]] for each t (parallel over t)."""
    st = np.ascontiguousarray(stations, dtype=np.int64)
    cl = np.ascontiguousarray(cells, dtype=np.int64)
    assert st.shape == cl.shape
    out = np.zeros(st.size)
    g, _z = geom._c()
    _load().gmo_entries(ctypes.byref(g), _ip(st), _ip(cl), st.size, _dp(out))
    return out


def dense(geom: Geometry) -> np.ndarray:
    """The full m x n matrix G (small geometries only)."""
    return rows(geom, np.arange(geom.m))


def forward(geom: Geometry, m, stations=None) -> np.ndarray:
    """d = G m (all stations, or the listed ones), summed in binary128."""
    mm = np.ascontiguousarray(m, dtype=np.float64).reshape(-1)
    assert mm.size == geom.n
    g, _z = geom._c()
    if stations is None:
        out = np.zeros(geom.m)
        _load().gmo_forward(ctypes.byref(g), _dp(mm), None, geom.m, _dp(out))
        return out.reshape(geom.sy, geom.sx)
    st = np.ascontiguousarray(stations, dtype=np.int64)
    out = np.zeros(st.size)
    _load().gmo_forward(ctypes.byref(g), _dp(mm), _ip(st), st.size, _dp(out))
    return out


def transpose(geom: Geometry, d, cells=None) -> np.ndarray:
    """m' = G^T d (all cells, or the listed ones), summed in binary128."""
    dd = np.ascontiguousarray(d, dtype=np.float64).reshape(-1)
    assert dd.size == geom.m
    g, _z = geom._c()
    if cells is None:
        out = np.zeros(geom.n)
        _load().gmo_transpose(ctypes.byref(g), _dp(dd), None, geom.n, _dp(out))
        return out.reshape(geom.nz, geom.ny, geom.nx)
    cl = np.ascontiguousarray(cells, dtype=np.int64)
    out = np.zeros(cl.size)
    _load().gmo_transpose(ctypes.byref(g), _dp(dd), _ip(cl), cl.size, _dp(out))
    return out


def threads() -> int:
    return _load().gmo_threads()


def set_threads(n: int) -> None:
    _load().gmo_set_threads(int(n))


def significand_bits() -> int:
    """Significand bits of the arithmetic the oracle runs in (113: IEEE binary128)."""
    return _load().gmo_mant_dig()
