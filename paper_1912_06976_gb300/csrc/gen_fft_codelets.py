"""Generates gm_fft_codelets.cuh: straight-line small DFTs for the register-resident FFT passes.

Each codelet dft<N>(v) transforms v[0..N-1] in place, natural order in and out,
forward (X_k = SUM_n x_n exp(-2 pi i n k / N)) or inverse (+i, unnormalised).
Odd primes use the symmetric-pair form (N-1)/2 real cosines and sines; 4 uses
the radix-4 butterfly; composite sizes are split N = N1 * N2 (Cooley-Tukey,
input n = N2 n1 + n2, output k = k1 + N1 k2) with the twiddles exp(-2 pi i
n2 k1 / N) emitted as literals; multiplications by +-1, +-i and (+-1 +- i)/sqrt2
are specialised.  Inputs known to be zero (the zero padding of the transforms)
are propagated symbolically, so the input-pruned variants dftN_inL skip the work
on them.  Constants are computed with mpmath at 40 digits, rounded to double and
written with 17 significant digits.

Run:  python gen_fft_codelets.py   (self-tests every codelet against numpy's FFT by executing
the emitted statements in Python, then rewrites gm_fft_codelets.cuh next to this file)
"""
import math
import os
import re

import mpmath

mpmath.mp.dps = 40


def cos2pi(k, n):
    return float(mpmath.cos(2 * mpmath.pi * k / n))


def sin2pi(k, n):
    return float(mpmath.sin(2 * mpmath.pi * k / n))

SIZES = [2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 15, 16, 18, 20, 21, 24, 25, 27, 28, 32, 35]

# preferred split of composite sizes (N1, N2)
SPLITS = {6: (2, 3), 8: (2, 4), 9: (3, 3), 10: (2, 5), 12: (4, 3), 14: (2, 7), 15: (3, 5), 16: (4, 4),
          18: (2, 9), 20: (4, 5), 21: (3, 7), 24: (8, 3), 25: (5, 5), 27: (3, 9), 28: (4, 7), 32: (4, 8), 35: (5, 7)}


def lit(x):
    if x == 0.0:
        return "R(0)"
    return f"R({x:.17g})"


class Emitter:
    def __init__(self):
        self.lines = []
        self.n = 0

    def tmp(self):
        self.n += 1
        return f"t{self.n}"

    def let(self, expr):
        t = self.tmp()
        self.lines.append(f"const R {t} = {expr};")
        return t

    # complex values are (re, im) pairs of expression names; None is an exact zero
    def add(self, a, b):
        if a is None:
            return b
        if b is None:
            return a
        return (self.let(f"{a[0]} + {b[0]}"), self.let(f"{a[1]} + {b[1]}"))

    def neg(self, a):
        if a is None:
            return None
        return (self.let(f"-{a[0]}"), self.let(f"-{a[1]}"))

    def sub(self, a, b):
        if b is None:
            return a
        if a is None:
            return self.neg(b)
        return (self.let(f"{a[0]} - {b[0]}"), self.let(f"{a[1]} - {b[1]}"))

    def mul_i(self, a, sign):
        """a * (sign * i)"""
        if a is None:
            return None
        return (self.let(f"-{a[1]}") if sign > 0 else a[1], a[0] if sign > 0 else self.let(f"-{a[0]}"))

    def scale(self, a, c):
        """a * real constant c (a complex)"""
        if a is None:
            return None
        return (f"{a[0]} * {lit(c)}", f"{a[1]} * {lit(c)}")

    def twiddle(self, a, k, n, sign):
        """a * exp(sign * 2 pi i k / n)"""
        if a is None:
            return None
        k %= n
        if k == 0:
            return a
        if 4 * k == n:
            return self.mul_i(a, sign)
        if 2 * k == n:
            return (self.let(f"-{a[0]}"), self.let(f"-{a[1]}"))
        if 4 * k == 3 * n:
            return self.mul_i(a, -sign)
        c = cos2pi(k, n)
        s = sign * sin2pi(k, n)
        if 8 * k % n == 0:  # odd multiples of pi/4: (c, s) = (+-h, +-h)
            h = lit(abs(c))
            # (x + i y)(c + i s) = (x c - y s) + i (x s + y c) with |c| = |s| = h
            sc, ss = (1 if c > 0 else -1), (1 if s > 0 else -1)
            re = self.let(f"({a[0]} {'-' if ss * sc > 0 else '+'} {a[1]}) * {lit(c)}")
            im = self.let(f"({a[0]} {'+' if ss * sc > 0 else '-'} {a[1]}) * {lit(s)}")
            del h
            return (re, im)
        return (self.let(f"{a[0]} * {lit(c)} - {a[1]} * {lit(s)}"),
                self.let(f"{a[0]} * {lit(s)} + {a[1]} * {lit(c)}"))

    def dft(self, x, sign):
        n = len(x)
        if n == 1:
            return list(x)
        if n == 2:
            return [self.add(x[0], x[1]), self.sub(x[0], x[1])]
        if n == 4:
            t0, t1 = self.add(x[0], x[2]), self.sub(x[0], x[2])
            t2, t3 = self.add(x[1], x[3]), self.sub(x[1], x[3])
            it3 = self.mul_i(t3, sign)
            return [self.add(t0, t2), self.add(t1, it3), self.sub(t0, t2), self.sub(t1, it3)]
        if n in SPLITS and math.gcd(*SPLITS[n]) == 1:
            # prime-factor (Good-Thomas) form for coprime n1, n2: inputs at (n2 a + n1 b) mod n,
            # DFT-n1 over a, DFT-n2 over b, output (k1, k2) at the CRT index
            # k = (n2 (n2^-1 mod n1) k1 + n1 (n1^-1 mod n2) k2) mod n -- no twiddle factors
            n1, n2 = SPLITS[n]
            t1, t2 = pow(n2, -1, n1), pow(n1, -1, n2)
            y = [self.dft([x[(n2 * a + n1 * b) % n] for a in range(n1)], sign) for b in range(n2)]
            out = [None] * n
            for k1 in range(n1):
                row = self.dft([y[b][k1] for b in range(n2)], sign)
                for k2 in range(n2):
                    out[(n2 * t1 * k1 + n1 * t2 * k2) % n] = row[k2]
            return out
        if n in SPLITS:
            n1, n2 = SPLITS[n]
            y = [[None] * n1 for _ in range(n2)]
            for b in range(n2):
                col = self.dft([x[n2 * a + b] for a in range(n1)], sign)
                for k1 in range(n1):
                    y[b][k1] = self.twiddle(col[k1], b * k1, n, sign)
            out = [None] * n
            for k1 in range(n1):
                row = self.dft([y[b][k1] for b in range(n2)], sign)
                for k2 in range(n2):
                    out[k1 + n1 * k2] = row[k2]
            return out
        # odd prime: symmetric pairs
        assert n % 2 == 1
        h = (n - 1) // 2
        a = [self.add(x[k], x[n - k]) for k in range(1, h + 1)]
        b = [self.sub(x[k], x[n - k]) for k in range(1, h + 1)]

        def lin(base, terms):
            """base + SUM c_k * t_k over the nonzero terms (base may be None)"""
            parts_r = ([base[0]] if base is not None else []) + [f"{t[0]} * {lit(c)}" for c, t in terms if t is not None]
            parts_i = ([base[1]] if base is not None else []) + [f"{t[1]} * {lit(c)}" for c, t in terms if t is not None]
            if not parts_r:
                return None
            return (self.let(" + ".join(parts_r)), self.let(" + ".join(parts_i)))

        out = [None] * n
        s0 = [x[0]] + a
        nz = [t for t in s0 if t is not None]
        out[0] = None if not nz else (self.let(" + ".join(t[0] for t in nz)), self.let(" + ".join(t[1] for t in nz)))
        for m in range(1, h + 1):
            A = lin(x[0], [(cos2pi(k * m, n), a[k - 1]) for k in range(1, h + 1)])
            B = lin(None, [(sin2pi(k * m, n), b[k - 1]) for k in range(1, h + 1)])
            # X_m = A + sign*i*B, X_{n-m} = A - sign*i*B
            iB = self.mul_i(B, sign)
            out[m] = self.add(A, iB)
            out[n - m] = self.sub(A, iB)
        return out


class CEmitter(Emitter):
    """The same DFT algorithms, emitted as operations on whole complex values (type C) through the
    cx_* helpers of the header prelude: one packed two-lane FP32 instruction per complex add,
    subtract, real scaling or real multiply-add when C = float2 (scalar code for double2)."""

    def let(self, expr):
        t = self.tmp()
        self.lines.append(f"const C {t} = {expr};")
        return t

    # complex values are names of C temporaries (or v[k]); None is an exact zero
    def add(self, a, b):
        if a is None:
            return b
        if b is None:
            return a
        return self.let(f"cx_add({a}, {b})")

    def neg(self, a):
        return None if a is None else self.let(f"cx_neg({a})")

    def sub(self, a, b):
        if b is None:
            return a
        if a is None:
            return self.neg(b)
        return self.let(f"cx_sub({a}, {b})")

    def mul_i(self, a, sign):
        if a is None:
            return None
        return self.let(f"cx_mul_i({a})" if sign > 0 else f"cx_mul_mi({a})")

    def twiddle(self, a, k, n, sign):
        if a is None:
            return None
        k %= n
        if k == 0:
            return a
        if 4 * k == n:
            return self.mul_i(a, sign)
        if 2 * k == n:
            return self.neg(a)
        if 4 * k == 3 * n:
            return self.mul_i(a, -sign)
        c = cos2pi(k, n)
        s = sign * sin2pi(k, n)
        if 8 * k % n == 0:  # odd multiples of pi/4: |c| = |s|
            mode = 1 if (c > 0) == (s > 0) else 0
            return self.let(f"cx_rot_diag({a}, {lit(c)}, {lit(s)}, {mode})")
        return self.let(f"cx_rot({a}, {lit(c)}, {lit(s)})")

    def dft(self, x, sign):
        n = len(x)
        if n in (1, 2, 4) or n in SPLITS:
            return Emitter.dft(self, x, sign)
        # odd prime: symmetric pairs, linear combinations as multiply-add chains
        h = (n - 1) // 2
        a = [self.add(x[k], x[n - k]) for k in range(1, h + 1)]
        b = [self.sub(x[k], x[n - k]) for k in range(1, h + 1)]

        def lin(base, terms):
            acc = base
            for c, t in terms:
                if t is None:
                    continue
                acc = self.let(f"cx_fma({t}, {lit(c)}, {acc})") if acc is not None else \
                    self.let(f"cx_scale({t}, {lit(c)})")
            return acc

        out = [None] * n
        acc = x[0]
        for t in a:
            acc = self.add(acc, t)
        out[0] = acc
        for m in range(1, h + 1):
            A = lin(x[0], [(cos2pi(k * m, n), a[k - 1]) for k in range(1, h + 1)])
            B = lin(None, [(sin2pi(k * m, n), b[k - 1]) for k in range(1, h + 1)])
            # X_m = A + sign*i*B, X_{n-m} = A - sign*i*B
            if B is None:
                out[m] = out[n - m] = A
            elif A is None:
                out[m] = self.mul_i(B, sign)
                out[n - m] = self.mul_i(B, -sign)
            else:
                out[m] = self.let(f"cx_addi({A}, {B}, {lit(float(sign))})")
                out[n - m] = self.let(f"cx_subi({A}, {B}, {lit(float(sign))})")
        return out


PRELUDE = r"""
// Complex helpers of the codelets: packed two-lane FP32 instructions for float2 (sm_100+), the
// same operations lane by lane for double2.  Each lane rounds exactly as the scalar form would.
__device__ __forceinline__ float2 cx_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 cx_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 cx_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 cx_mul_i(float2 a) { return make_float2(-a.y, a.x); }
__device__ __forceinline__ float2 cx_mul_mi(float2 a) { return make_float2(a.y, -a.x); }
__device__ __forceinline__ float2 cx_scale(float2 a, float c) { return __fmul2_rn(a, make_float2(c, c)); }
__device__ __forceinline__ float2 cx_fma(float2 t, float c, float2 acc) { return __ffma2_rn(t, make_float2(c, c), acc); }
__device__ __forceinline__ float2 cx_rot(float2 a, float c, float s) {
    return __ffma2_rn(make_float2(a.y, a.x), make_float2(-s, s), __fmul2_rn(a, make_float2(c, c)));
}
// (x + i y)(c + i s) with |c| = |s|: mode 1 -> ((x - y) c, (x + y) s), mode 0 -> ((x + y) c, (x - y) s)
__device__ __forceinline__ float2 cx_rot_diag(float2 a, float c, float s, int mode) {
    const float2 u = __ffma2_rn(make_float2(a.y, a.y), mode ? make_float2(-1.f, 1.f) : make_float2(1.f, -1.f),
                                make_float2(a.x, a.x));
    return __fmul2_rn(u, make_float2(c, s));
}
// A + sign i B and A - sign i B
__device__ __forceinline__ float2 cx_addi(float2 A, float2 B, float sign) {
    return __ffma2_rn(make_float2(B.y, B.x), make_float2(-sign, sign), A);
}
__device__ __forceinline__ float2 cx_subi(float2 A, float2 B, float sign) {
    return __ffma2_rn(make_float2(B.y, B.x), make_float2(sign, -sign), A);
}

__device__ __forceinline__ double2 cx_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cx_sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cx_neg(double2 a) { return make_double2(-a.x, -a.y); }
__device__ __forceinline__ double2 cx_mul_i(double2 a) { return make_double2(-a.y, a.x); }
__device__ __forceinline__ double2 cx_mul_mi(double2 a) { return make_double2(a.y, -a.x); }
__device__ __forceinline__ double2 cx_scale(double2 a, double c) { return make_double2(a.x * c, a.y * c); }
__device__ __forceinline__ double2 cx_fma(double2 t, double c, double2 acc) {
    return make_double2(fma(t.x, c, acc.x), fma(t.y, c, acc.y));
}
__device__ __forceinline__ double2 cx_rot(double2 a, double c, double s) {
    return make_double2(fma(-a.y, s, a.x * c), fma(a.x, s, a.y * c));
}
__device__ __forceinline__ double2 cx_rot_diag(double2 a, double c, double s, int mode) {
    return mode ? make_double2((a.x - a.y) * c, (a.x + a.y) * s) : make_double2((a.x + a.y) * c, (a.x - a.y) * s);
}
__device__ __forceinline__ double2 cx_addi(double2 A, double2 B, double sign) {
    return make_double2(fma(-sign, B.y, A.x), fma(sign, B.x, A.y));
}
__device__ __forceinline__ double2 cx_subi(double2 A, double2 B, double sign) {
    return make_double2(fma(sign, B.y, A.x), fma(-sign, B.x, A.y));
}
"""


def codelet(n, inverse, nin=None):
    """DFT-n on v[0..n-1]; with nin < n the inputs v[nin..n-1] are taken as zero (not read)."""
    nin = n if nin is None else nin
    e = CEmitter()
    x = [f"v[{k}]" if k < nin else None for k in range(n)]
    out = e.dft(x, +1 if inverse else -1)
    body = ["    " + ln for ln in e.lines]
    body += [f"    v[{k}] = {out[k] if out[k] else 'C{}'};" for k in range(n)]
    name = ("idft" if inverse else "dft") + str(n) + ("" if nin == n else f"_in{nin}")
    return (f"template <typename C>\n__device__ __forceinline__ void {name}(C (&v)[{n}]) {{\n"
            f"    using R = typename real_of<C>::type;\n" + "\n".join(body) + "\n}\n")


# input-pruned variants: sizes used as the first pass of zero-padded transforms, with the
# numbers of leading nonzero inputs offered (a kernel picks the smallest bucket that covers it)
# (none instantiated: in a trial the pruned first passes saved about 5% of the arithmetic of the
# prime-radix codelets and ran slower than the full codelets)
PRUNED = {}


def selftest():
    """Executes every emitted codelet body in Python (complex numbers standing in for C and the
    cx_* helpers written out) and compares it with numpy's FFT."""
    import numpy as np

    helpers = {
        "cx_add": lambda a, b: a + b, "cx_sub": lambda a, b: a - b, "cx_neg": lambda a: -a,
        "cx_mul_i": lambda a: 1j * a, "cx_mul_mi": lambda a: -1j * a, "cx_scale": lambda a, c: a * c,
        "cx_fma": lambda t, c, acc: acc + c * t, "cx_rot": lambda a, c, s: a * complex(c, s),
        "cx_rot_diag": lambda a, c, s, mode: (complex((a.real - a.imag) * c, (a.real + a.imag) * s) if mode
                                              else complex((a.real + a.imag) * c, (a.real - a.imag) * s)),
        "cx_addi": lambda A, B, sg: A + sg * 1j * B, "cx_subi": lambda A, B, sg: A - sg * 1j * B,
    }
    rng = np.random.default_rng(0)
    worst = 0.0
    cases = [(n, n) for n in SIZES] + [(n, L) for n, ls in PRUNED.items() for L in ls]
    for n, nin in cases:
        for inv in (False, True):
            e = CEmitter()
            out = e.dft([f"v[{k}]" if k < nin else None for k in range(n)], +1 if inv else -1)
            code = [re.sub(r"R\(([^)]*)\)", r"\1", ln.replace("const C ", "")).rstrip(";") for ln in e.lines]
            x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
            x[nin:] = 0
            env = dict(helpers, v=list(x))
            exec("\n".join(code), env)
            got = np.array([eval(o, env) if o else 0j for o in out])
            ref = np.fft.ifft(x) * n if inv else np.fft.fft(x)
            err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
            worst = max(worst, err)
            assert err < 1e-14, (n, nin, inv, err)
    return worst


def render() -> str:
    """The text of gm_fft_codelets.cuh."""
    parts = ["// gm_fft_codelets.cuh -- GENERATED by gen_fft_codelets.py; do not edit by hand.",
             "// Straight-line in-register DFTs, natural order: dftN (forward, exp(-2 pi i nk/N)) and",
             "// idftN (inverse, exp(+2 pi i nk/N), unnormalised), for C = float2 or double2.",
             "#pragma once", "", "#include <cuda_runtime.h>", "", "#include \"gm_common.cuh\"", "", "namespace gm {", "namespace cl {", PRELUDE]
    for n in SIZES:
        parts.append(codelet(n, False))
        parts.append(codelet(n, True))
    for n, ls in PRUNED.items():
        for L in ls:
            parts.append(codelet(n, False, L))
            parts.append(codelet(n, True, L))
    parts.append("// Dispatch by size: Dft<N, INV>::run(v); DftIn<N, L, INV>::run(v) reads only v[0..L-1].")
    parts.append("template <int N, bool INV> struct Dft;")
    for n in SIZES:
        for inv in (False, True):
            nm = ("idft" if inv else "dft") + str(n)
            parts.append(f"template <> struct Dft<{n}, {'true' if inv else 'false'}> {{ template <typename C> "
                         f"__device__ __forceinline__ static void run(C (&v)[{n}]) {{ {nm}(v); }} }};")
    parts.append("template <int N, int L, bool INV> struct DftIn { template <typename C> "
                 "__device__ __forceinline__ static void run(C (&v)[N]) { Dft<N, INV>::run(v); } };")
    for n, ls in PRUNED.items():
        for L in ls:
            for inv in (False, True):
                nm = ("idft" if inv else "dft") + f"{n}_in{L}"
                parts.append(f"template <> struct DftIn<{n}, {L}, {'true' if inv else 'false'}> {{ template <typename C> "
                             f"__device__ __forceinline__ static void run(C (&v)[{n}]) {{ {nm}(v); }} }};")
    parts += ["", "}  // namespace cl", "}  // namespace gm", ""]
    return "\n".join(parts)


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gm_fft_codelets.cuh")
    with open(out, "w") as f:
        f.write(render())
    print(out)


if __name__ == "__main__":
    print("self-test: worst relative error", selftest())
    main()
