"""The C ABI on the host (no GPU needed): the library builds and loads, exports
every function the headers under include/ declare, and its host-only logic (FFT
length choice, parameter validation, no-device behaviour) is right."""
import ctypes
import glob
import os
import re

import pytest

from paper_1912_06976_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    from paper_1912_06976_gb300 import gravmag

    return gravmag


def _declared_functions(header=None):
    names = []
    for path in sorted(glob.glob(os.path.join(ROOT, "include", header or "*.h"))):
        txt = re.sub(r"/\*.*?\*/", "", open(path).read(), flags=re.S)
        names += re.findall(r"^GM_API\s+[\w\s\*]*?\b(\w+)\s*\(", txt, flags=re.M)
    return names


def test_header_declares_the_boundary():
    names = _declared_functions("gravmag.h")
    for required in ("grav_mag_setup", "grav_mag_setup_ex", "apply_forward", "apply_transpose",
                     "apply_forward_host", "apply_transpose_host", "apply_forward_host_async",
                     "apply_transpose_host_async", "grav_mag_destroy", "gm_status_string", "gm_cgls",
                     "gm_cgls_noalloc"):
        assert required in names
    net = _declared_functions("gm_warmstart.h")
    for required in ("gm_net_create", "gm_net_forward", "gm_net_train_step", "gm_net_get_params"):
        assert required in net


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(B.LIB)
    missing = [n for n in _declared_functions() if not hasattr(so, n)]
    assert not missing, missing


def _smooth_even(n):
    m = max(n, 2)
    while True:
        if m % 2 == 0:
            k = m
            for p in (2, 3, 5, 7):
                while k % p == 0:
                    k //= p
            if k == 1:
                return m
        m += 1


def test_fft_length_is_smallest_even_7_smooth(lib):
    for n in list(range(1, 300)) + [549, 659, 1000, 2047, 4097]:
        assert lib.fft_length(n) == _smooth_even(n)
    assert lib.fft_length(659) == 672 and lib.fft_length(549) == 560  # the 300x250 grid, 10 % padding
    assert lib.fft_length(0) == -1


@pytest.mark.parametrize("field,value", [("sx", 0), ("nz", 0), ("pxl", -1), ("dx", 0.0), ("dy", -1.0),
                                         ("kind", 7), ("precision", 3)])
def test_validate_rejects_bad_fields(lib, field, value):
    p, keep = lib.make_params(8, 8, 4, 10.0, 10.0, 10.0)
    lib.validate(p)
    setattr(p, field, value)
    with pytest.raises(lib.GravMagError) as e:
        lib.validate(p)
    assert e.value.status == lib.GM_EINVAL


def test_validate_magnetic_angles_and_zplanes(lib):
    p, keep = lib.make_params(8, 8, 2, 10.0, 10.0, kind=lib.MAGNETIC, incl_deg=91.0, zplanes=[0, 5, 9])
    with pytest.raises(lib.GravMagError):
        lib.validate(p)
    p, keep = lib.make_params(8, 8, 2, 10.0, 10.0, kind=lib.MAGNETIC, incl_deg=60.0, zplanes=[0, 5, 5])
    with pytest.raises(lib.GravMagError):
        lib.validate(p)
    p, keep = lib.make_params(8, 8, 2, 10.0, 10.0, kind=lib.MAGNETIC, incl_deg=60.0, zplanes=[2, 5, 9])
    lib.validate(p)
    p, keep = lib.make_params(3000, 8, 2, 10.0, 10.0, 10.0)  # 2*3000-1 > the single-CTA FFT limit
    with pytest.raises(lib.GravMagError):
        lib.validate(p)


def test_status_strings(lib):
    so = lib.load()
    for s in range(7):
        assert so.gm_status_string(s).startswith(b"GM_")


def test_setup_without_a_device_fails_cleanly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    so = lib.load()
    h = so.grav_mag_setup(8, 8, 2, 10.0, 10.0, 10.0, 0, 0, 0, 0.0, 0.0)
    assert not h
    assert so.gm_last_status() == lib.GM_ENODEV
    assert so.apply_forward(None, None, None, None) == lib.GM_EINVAL
    assert so.grav_mag_destroy(None) == lib.GM_OK


def test_operator_entry_points_reject_a_null_handle_before_touching_a_device(lib):
    """Every call on a handle checks it first: a NULL handle is GM_EINVAL with a message, on any
    machine, with or without a GPU."""
    import ctypes

    so = lib.load()
    buf = (ctypes.c_float * 16)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    for fn in ("apply_forward", "apply_transpose", "apply_forward_host", "apply_transpose_host",
               "apply_forward_host_async", "apply_transpose_host_async"):
        assert getattr(so, fn)(None, p, p, None) == lib.GM_EINVAL, fn
        assert so.gm_last_status() == lib.GM_EINVAL
        assert so.gm_last_error()
    assert so.gm_cgls(None, p, None, p, 0.1, 3, None, None) == lib.GM_EINVAL
    assert so.gm_cgls_noalloc(None, p, None, p, 0.1, 3, None, None) == lib.GM_EINVAL


def test_network_rejects_bad_arguments_without_a_device(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1912_06976_gb300 import warmstart

    so = warmstart._lib()
    assert not so.gm_net_create(40, 16, 4, 0)  # grid not a multiple of 16
    assert not so.gm_net_create(64, 8, 4, 0)   # depth other than 16
    assert not so.gm_net_create(64, 16, 0, 0)  # empty batch
    assert not so.gm_net_create(64, 16, 4, 0)  # valid, but no device
    assert b"device" in so.gm_net_last_error()
    assert so.gm_net_forward(None, None, None, 1, None) == lib.GM_EINVAL
    assert so.gm_net_train_step(None, None, None, 1, None, 1, 0.0, None, None) == lib.GM_EINVAL
    assert so.gm_net_num_params(None) == -1
    assert so.gm_net_destroy(None) == lib.GM_OK
