"""CPU checks of the straight-line DFT codelets that every FFT pass of the apply kernels runs.

The header gm_fft_codelets.cuh is generated by gen_fft_codelets.py.  These tests execute each
emitted codelet body in Python (complex numbers in place of the CUDA types) against numpy's
FFT, forward and inverse, and check that the committed header is exactly what the generator
emits, so the kernels compile the codelets that were checked.
"""
import os
import sys

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1912_06976_gb300", "csrc")


@pytest.fixture(scope="module")
def gen():
    pytest.importorskip("mpmath")
    sys.path.insert(0, CSRC)
    try:
        import gen_fft_codelets as g
    finally:
        sys.path.remove(CSRC)
    return g


def test_every_codelet_is_the_dft(gen):
    # worst relative error over all sizes, both directions, random complex inputs
    assert gen.selftest() < 1e-14


def test_committed_header_is_the_generator_output(gen):
    with open(os.path.join(CSRC, "gm_fft_codelets.cuh")) as f:
        assert f.read() == gen.render()


def test_codelet_sizes_cover_every_ladder_radix(gen):
    # every radix named by the row and column ladders has a codelet
    import re

    with open(os.path.join(CSRC, "gm_fast_ops.h")) as f:
        text = f.read()
    radices = set()
    for n, a, b in re.findall(r"F\((\d+), (\d+), (\d+)\)", text):
        assert int(a) * int(b) == int(n), (n, a, b)
        radices.update((int(a), int(b)))
    # the FP32 row table's own split of 672
    radices.update((24, 28))
    assert radices <= set(gen.SIZES), sorted(radices - set(gen.SIZES))


def test_embedded_constants_are_the_twiddle_values(gen):
    # the cosines and sines the codelets embed, against an extended-precision evaluation
    # (long double: 64-bit significand on x86-64, 113-bit on aarch64) rounded to double
    pi = np.longdouble("3.14159265358979323846264338327950288")
    for n in gen.SIZES:
        for k in range(n):
            a = np.longdouble(2) * pi * k / n
            c, s_ = float(np.cos(a)), float(np.sin(a))
            assert abs(gen.cos2pi(k, n) - c) <= np.spacing(abs(c)) + 1e-18, (k, n)
            assert abs(gen.sin2pi(k, n) - s_) <= np.spacing(abs(s_)) + 1e-18, (k, n)
