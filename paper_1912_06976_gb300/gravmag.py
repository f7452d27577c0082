"""Python binding of the C ABI in include/gravmag.h (argument marshalling only).

Every product, set-up step and CGLS iteration runs in the CUDA library
``_build/libgravmag.so``; this module checks tensors (device, dtype, shape,
contiguity), passes their device pointers and the current CUDA stream through
ctypes, and turns status codes into exceptions.  There is no CPU fallback: if
the library is missing or fails to load, ``load()`` raises.

Layouts follow Sec. 2 of Hogue, Renaut & Vatankhah (arXiv 1912.06976), Eqs.
Gslice / htilde: a model is ``m[nz, ny, nx]`` and data are ``d[sy, sx]`` (x
fastest).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

GRAVITY = 0
MAGNETIC = 1
F32 = 0
F64 = 1
DF64 = 2  # FP64 vectors, arithmetic on pairs of FP32 values (see include/gravmag.h)

GM_OK, GM_EINVAL, GM_ENOMEM, GM_ECUDA, GM_ETIMEOUT, GM_EDEVICE, GM_ENODEV = range(7)
_STATUS_NAMES = ["GM_OK", "GM_EINVAL", "GM_ENOMEM", "GM_ECUDA", "GM_ETIMEOUT", "GM_EDEVICE", "GM_ENODEV"]


class GravMagError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        name = _STATUS_NAMES[status] if 0 <= status < len(_STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


class Params(ctypes.Structure):
    """Mirror of gm_params."""

    _fields_ = [
        ("sx", ctypes.c_int), ("sy", ctypes.c_int), ("nz", ctypes.c_int),
        ("pxl", ctypes.c_int), ("pxr", ctypes.c_int), ("pyl", ctypes.c_int), ("pyr", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("zplanes", ctypes.POINTER(ctypes.c_double)),
        ("kind", ctypes.c_int),
        ("incl_deg", ctypes.c_double), ("decl_deg", ctypes.c_double), ("F_nT", ctypes.c_double),
        ("precision", ctypes.c_int),
    ]


class Info(ctypes.Structure):
    """Mirror of gm_info."""

    _fields_ = [
        ("sx", ctypes.c_int), ("sy", ctypes.c_int), ("nz", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("fft_nx", ctypes.c_int), ("fft_ny", ctypes.c_int), ("spec_nx", ctypes.c_int),
        ("kind", ctypes.c_int), ("precision", ctypes.c_int),
        ("n_model", ctypes.c_int64), ("n_data", ctypes.c_int64),
        ("spectrum_bytes", ctypes.c_size_t), ("workspace_bytes", ctypes.c_size_t),
        ("setup_ms", ctypes.c_double), ("spectrum_real", ctypes.c_int),
    ]


class KernelTime(ctypes.Structure):
    """Mirror of gm_kernel_time."""

    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int), ("total_ms", ctypes.c_double)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load():
    """Loads libgravmag.so (built by ``build.build()`` / ``__graft_entry__.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build the CUDA library first (paper_1912_06976_gb300.build)")
        lib = ctypes.CDLL(path)
        vp, c_int, c_double, c_size_t = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        sig = {
            "grav_mag_setup": (vp, [c_int, c_int, c_int, c_double, c_double, c_double, c_int, c_int, c_int,
                                    c_double, c_double]),
            "grav_mag_setup_ex": (vp, [ctypes.POINTER(Params)]),
            "apply_forward": (c_int, [vp, vp, vp, vp]),
            "apply_transpose": (c_int, [vp, vp, vp, vp]),
            "apply_forward_host": (c_int, [vp, vp, vp, vp]),
            "apply_transpose_host": (c_int, [vp, vp, vp, vp]),
            "apply_forward_host_async": (c_int, [vp, vp, vp, vp]),
            "apply_transpose_host_async": (c_int, [vp, vp, vp, vp]),
            "grav_mag_destroy": (c_int, [vp]),
            "gm_get_info": (c_int, [vp, ctypes.POINTER(Info)]),
            "gm_copy_spectrum": (c_int, [vp, vp, c_size_t]),
            "gm_fft_length": (c_int, [c_int]),
            "gm_validate_params": (c_int, [ctypes.POINTER(Params)]),
            "gm_set_memory_limit": (None, [c_size_t]),
            "gm_cgls": (c_int, [vp, vp, vp, vp, c_double, c_int, ctypes.POINTER(c_double), vp]),
            "gm_last_status": (c_int, []),
            "gm_last_error": (ctypes.c_char_p, []),
            "gm_status_string": (ctypes.c_char_p, [c_int]),
            "gm_last_launch_count": (c_int, [vp]),
            "gm_enable_timing": (c_int, [vp, c_int]),
            "gm_cgls_noalloc": (c_int, [vp, vp, vp, vp, c_double, c_int, ctypes.POINTER(c_double), vp]),
            "gm_cgls_noalloc_capacity": (c_size_t, []),
            "gm_kernel_times": (c_int, [vp, ctypes.POINTER(KernelTime), c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(status):
    if status != GM_OK:
        raise GravMagError(status, load().gm_last_error().decode(errors="replace"))


def fft_length(n: int) -> int:
    return load().gm_fft_length(int(n))


def validate(params: Params) -> None:
    _check(load().gm_validate_params(ctypes.byref(params)))


def set_memory_limit(nbytes: int) -> None:
    load().gm_set_memory_limit(int(nbytes))


def make_params(sx, sy, nz, dx, dy, dz=None, *, px=0, py=0, pxr=None, pyr=None, zplanes=None, kind=GRAVITY,
                incl_deg=90.0, decl_deg=0.0, F_nT=50000.0, precision=F32):
    """A gm_params record; returns (params, keepalive) -- keep the second alive while using the first."""
    z = None
    if zplanes is not None:
        z = np.ascontiguousarray(zplanes, dtype=np.float64)
        zp = z.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    else:
        zp = ctypes.POINTER(ctypes.c_double)()
    p = Params(int(sx), int(sy), int(nz), int(px), int(px if pxr is None else pxr), int(py),
               int(py if pyr is None else pyr), float(dx), float(dy), float(dz if dz is not None else 0.0), zp,
               int(kind), float(incl_deg), float(decl_deg), float(F_nT), int(precision))
    return p, z


def _stream_ptr(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Operator:
    """The fast operator G of one geometry: ``forward(m) = G m``, ``transpose(d) = G^T d``.

    Wraps one C-ABI handle (spectra and workspace live on the GPU that is
    current at construction).  ``precision`` is F32, F64 or DF64; tensors passed
    in must be CUDA tensors of the matching dtype (float32 for F32, float64 otherwise).
    """

    def __init__(self, sx, sy, nz, dx, dy, dz=None, *, px=0, py=0, pxr=None, pyr=None, zplanes=None,
                 kind=GRAVITY, incl_deg=90.0, decl_deg=0.0, F_nT=50000.0, precision=F32):
        lib = load()
        self._params, self._keep = make_params(sx, sy, nz, dx, dy, dz, px=px, py=py, pxr=pxr, pyr=pyr,
                                               zplanes=zplanes, kind=kind, incl_deg=incl_deg, decl_deg=decl_deg,
                                               F_nT=F_nT, precision=precision)
        h = lib.grav_mag_setup_ex(ctypes.byref(self._params))
        if not h:
            _check(lib.gm_last_status())
            raise GravMagError(GM_ECUDA, "setup returned NULL")
        self._h = ctypes.c_void_p(h)
        self.info = self.get_info()
        self.precision = precision

    @classmethod
    def from_workload(cls, w, precision=F32):
        return cls(w.sx, w.sy, w.nz, w.dx, w.dy, w.dz, px=w.pxl, py=w.pyl, pxr=w.pxr, pyr=w.pyr, kind=w.kind,
                   incl_deg=w.incl_deg, decl_deg=w.decl_deg, F_nT=w.F_nT, precision=precision)

    @property
    def handle(self):
        return self._h

    @property
    def dtype(self):
        import torch

        return torch.float32 if self.precision == F32 else torch.float64

    @property
    def model_shape(self):
        return (self.info.nz, self.info.ny, self.info.nx)

    @property
    def data_shape(self):
        return (self.info.sy, self.info.sx)

    def get_info(self) -> Info:
        inf = Info()
        _check(load().gm_get_info(self._h, ctypes.byref(inf)))
        return inf

    def _arg(self, t, n):
        import torch

        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError("expected a CUDA tensor")
        if t.dtype != self.dtype:
            raise TypeError(f"expected dtype {self.dtype}, got {t.dtype}")
        if t.numel() != n:
            raise ValueError(f"expected {n} elements, got {t.numel()}")
        if not t.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return ctypes.c_void_p(t.data_ptr())

    def forward(self, m, out=None, stream=None):
        """d = G m (Algorithm multbttb, t = 1)."""
        import torch

        if out is None:
            out = torch.empty(self.data_shape, dtype=self.dtype, device=m.device)
        _check(load().apply_forward(self._h, self._arg(m, self.info.n_model), self._arg(out, self.info.n_data),
                                    _stream_ptr(stream)))
        return out

    def transpose(self, d, out=None, stream=None):
        """m' = G^T d (Algorithm multbttb, t = 2)."""
        import torch

        if out is None:
            out = torch.empty(self.model_shape, dtype=self.dtype, device=d.device)
        _check(load().apply_transpose(self._h, self._arg(d, self.info.n_data), self._arg(out, self.info.n_model),
                                      _stream_ptr(stream)))
        return out

    def _host_arg(self, a, n):
        import torch

        if isinstance(a, torch.Tensor):
            if a.is_cuda or a.dtype != self.dtype or a.numel() != n or not a.is_contiguous():
                raise TypeError("expected a contiguous CPU tensor of the operator's dtype")
            return ctypes.c_void_p(a.data_ptr())
        raise TypeError("expected a torch CPU tensor")

    def forward_host(self, m_host, out_host, stream=None):
        """d = G m with host tensors (copies inside; synchronises)."""
        _check(load().apply_forward_host(self._h, self._host_arg(m_host, self.info.n_model),
                                         self._host_arg(out_host, self.info.n_data), _stream_ptr(stream)))
        return out_host

    def transpose_host(self, d_host, out_host, stream=None):
        """m' = G^T d with host tensors (copies inside; synchronises)."""
        _check(load().apply_transpose_host(self._h, self._host_arg(d_host, self.info.n_data),
                                           self._host_arg(out_host, self.info.n_model), _stream_ptr(stream)))
        return out_host

    def forward_host_async(self, m_host, out_host, stream=None):
        """d = G m with host tensors, enqueued on `stream` without waiting: out_host is complete
        once the stream has been synchronised; both tensors must stay alive until then."""
        _check(load().apply_forward_host_async(self._h, self._host_arg(m_host, self.info.n_model),
                                               self._host_arg(out_host, self.info.n_data), _stream_ptr(stream)))
        return out_host

    def transpose_host_async(self, d_host, out_host, stream=None):
        """m' = G^T d with host tensors, enqueued on `stream` without waiting (see forward_host_async)."""
        _check(load().apply_transpose_host_async(self._h, self._host_arg(d_host, self.info.n_data),
                                                 self._host_arg(out_host, self.info.n_model), _stream_ptr(stream)))
        return out_host

    def spectrum(self) -> np.ndarray:
        """The stored spectra as complex numpy array [spec_nx, nz, fft_ny]."""
        inf = self.info
        dt = np.complex64 if self.precision == F32 else np.complex128
        out = np.empty((inf.spec_nx, inf.nz, inf.fft_ny), dtype=dt)
        _check(load().gm_copy_spectrum(self._h, ctypes.c_void_p(out.ctypes.data), out.nbytes))
        return out

    def cgls(self, d, alpha, iters, x0=None, out=None, stream=None, residuals=True):
        """Tikhonov CGLS on the device; returns (x, ||G x_k - d|| for k = 0..iters or None)."""
        import torch

        if out is None:
            out = torch.empty(self.model_shape, dtype=self.dtype, device=d.device)
        res = (ctypes.c_double * (iters + 1))() if residuals else None
        x0p = self._arg(x0, self.info.n_model) if x0 is not None else ctypes.c_void_p(0)
        _check(load().gm_cgls(self._h, self._arg(d, self.info.n_data), x0p, self._arg(out, self.info.n_model),
                              float(alpha), int(iters), res, _stream_ptr(stream)))
        return out, (np.array(res[:]) if residuals else None)

    def cgls_noalloc(self, d, alpha, iters, out, x0=None, stream=None, residuals=True):
        """Like cgls(), through the entry point that allocates no device memory (its scratch is a
        fixed array inside the library); the caller passes the output tensor."""
        res = (ctypes.c_double * (iters + 1))() if residuals else None
        x0p = self._arg(x0, self.info.n_model) if x0 is not None else ctypes.c_void_p(0)
        _check(load().gm_cgls_noalloc(self._h, self._arg(d, self.info.n_data), x0p,
                                      self._arg(out, self.info.n_model), float(alpha), int(iters), res,
                                      _stream_ptr(stream)))
        return out, (np.array(res[:]) if residuals else None)

    def last_launch_count(self) -> int:
        return load().gm_last_launch_count(self._h)

    def enable_timing(self, capacity: int) -> None:
        """Bracket up to `capacity` of this handle's launches with CUDA events (0 disables)."""
        _check(load().gm_enable_timing(self._h, int(capacity)))

    def kernel_times(self) -> dict:
        """{kernel name: (launches, total device ms)} since the last call; resets the counters."""
        buf = (KernelTime * 16)()
        k = load().gm_kernel_times(self._h, buf, 16)
        if k < 0:
            _check(load().gm_last_status())
        return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms) for i in range(k)}

    def close(self):
        if getattr(self, "_h", None):
            _check(load().grav_mag_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_function():
    import torch

    class GravMagFunction(torch.autograd.Function):
        """d = G m with the transpose product as its hand-written backward: grad_m = G^T grad_d."""

        @staticmethod
        def forward(ctx, m, op):
            ctx.op = op
            return op.forward(m.contiguous())

        @staticmethod
        def backward(ctx, grad_d):
            return ctx.op.transpose(grad_d.contiguous()), None

    return GravMagFunction


_fn = None


def gravmag_apply(m, op: Operator):
    """Differentiable d = G m (torch.autograd); backward runs the transpose kernels."""
    global _fn
    if _fn is None:
        _fn = _autograd_function()
    return _fn.apply(m, op)


def rel_err(x, ref) -> float:
    """Relative 2-norm error ||x - ref|| / ||ref|| (complex inputs keep their imaginary parts)."""
    x, ref = np.asarray(x), np.asarray(ref)
    dt = np.complex128 if (np.iscomplexobj(x) or np.iscomplexobj(ref)) else np.float64
    x, ref = x.astype(dt).ravel(), ref.astype(dt).ravel()
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))


__all__ = ["Operator", "gravmag_apply", "load", "fft_length", "validate", "make_params", "set_memory_limit",
           "GravMagError", "GRAVITY", "MAGNETIC", "F32", "F64", "DF64"]
