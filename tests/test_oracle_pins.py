"""Pins of the CPU oracle to facts other than itself (no GPU).

Each test ties the oracle (oracle/gm_oracle.c) to something the paper or the
mathematics fixes independently: closed-form limits, brute-force quadrature of
the integrand definitions, exact additivity, Laplace's equation, the
structural statements of Sec. 2.2 (Toeplitz / symmetry / worked examples) and
the sizes printed in Table 1.  A dropped term, a wrong sign, a wrong
coefficient or a transposed index in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

import oracle as O
from tests.conftest import rel_err

GAMMA = 6.67430e-3  # mGal per (g/cm^3 m): G = 6.67430e-11 SI, 1 g/cm^3 = 1e3 kg/m^3, 1 m/s^2 = 1e5 mGal


def _gl3(f, bounds, n=24, sub=2):
    """Composite tensor Gauss-Legendre integral of f(X, Y, Z) over a box."""
    x, w = leggauss(n)
    (x1, x2), (y1, y2), (z1, z2) = bounds
    ex, ey, ez = (np.linspace(a, b, sub + 1) for a, b in ((x1, x2), (y1, y2), (z1, z2)))
    tot = 0.0
    for a in range(sub):
        for b in range(sub):
            for c in range(sub):
                hx, hy, hz = ex[a + 1] - ex[a], ey[b + 1] - ey[b], ez[c + 1] - ez[c]
                xs = hx / 2 * x + (ex[a + 1] + ex[a]) / 2
                ys = hy / 2 * x + (ey[b + 1] + ey[b]) / 2
                zs = hz / 2 * x + (ez[c + 1] + ez[c]) / 2
                W = np.einsum("i,j,k->ijk", w, w, w) * hx * hy * hz / 8
                X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
                tot += np.sum(W * f(X, Y, Z))
    return tot


def _fhat(incl_deg, decl_deg):
    I, D = math.radians(incl_deg), math.radians(decl_deg)
    return np.array([math.cos(I) * math.cos(D), math.cos(I) * math.sin(D), math.sin(I)])


def _dipole_integrand(fh):
    """F^ . (grad grad 1/r) . F^ at relative position (X, Y, Z) (x North, y East, z down)."""

    def f(X, Y, Z):
        r2 = X * X + Y * Y + Z * Z
        r5 = r2 * r2 * np.sqrt(r2)
        comps = (X, Y, Z)
        s = 0.0
        for a in range(3):
            for b in range(3):
                s = s + fh[a] * fh[b] * (3.0 * comps[a] * comps[b] - (r2 if a == b else 0.0)) / r5
        return s

    return f


def _cell_bounds(geom, i, j, p, q, r):
    """Cell (p,q,r) relative to station (i,j), from the geometry of Sec. 2.1.2:
    cells start at 0, the station sits at the centre of unpadded cell (i,j)."""
    a = (i + geom.pxl + 0.5) * geom.dx
    b = (j + geom.pyl + 0.5) * geom.dy
    return ((p * geom.dx - a, (p + 1) * geom.dx - a),
            (q * geom.dy - b, (q + 1) * geom.dy - b),
            (geom.zplanes[r], geom.zplanes[r + 1]))


# ---------------------------------------------------------------- P1 point mass
@pytest.mark.parametrize("c", [(0.0, 0.0, 1000.0), (300.0, -200.0, 800.0), (-1500.0, 700.0, 90.0)])
def test_point_mass_limit_gravity(c):
    """A small cube far away attracts like a point mass gamma*rho*V*z/r^3 (Sec. 4.1 units)."""
    a = 5.0
    g = GAMMA * O.prism_grav(c[0] - a, c[0] + a, c[1] - a, c[1] + a, c[2] - a, c[2] + a)
    r = math.sqrt(sum(t * t for t in c))
    assert g == pytest.approx(GAMMA * (2 * a) ** 3 * c[2] / r ** 3, rel=1e-6)


def test_point_mass_limit_through_grid_entry():
    """Same limit through the grid indexing: a 1 m cell 100 m below and 120 m / 40 m aside."""
    geom = O.Geometry(1, 1, 2, 1.0, 1.0, (0.0, 100.0, 101.0), 0, 300, 0, 300, O.GRAVITY)
    e = O.entry(geom, 0, 0, 120, 40, 1)
    x, y, z = 120.0, 40.0, 100.5  # cell centre relative to the station at (0.5, 0.5, 0)
    r = math.sqrt(x * x + y * y + z * z)
    assert e == pytest.approx(GAMMA * z / r ** 3, rel=1e-6)


# ---------------------------------------------------------------- P2 Bouguer slab
def test_bouguer_slab_limit():
    """A wide horizontal slab tends to 2 pi gamma rho dz; a square of half-width L at mean
    depth zbar falls short by a relative amount between 0.5 zbar/L and zbar/L (a disc of
    radius L falls short by about zbar/L)."""
    dz, zbar = 10.0, 55.0
    for L in (1e3, 1e4, 1e5):
        g = O.prism_grav(-L, L, -L, L, zbar - dz / 2, zbar + dz / 2)
        deficit = (2 * math.pi * dz - g) / (2 * math.pi * dz)
        assert 0.5 * zbar / L < deficit < zbar / L


# ---------------------------------------------------------------- P3 additivity
def _split8(x1, x2, y1, y2, z1, z2):
    xm, ym, zm = (x1 + x2) / 2, (y1 + y2) / 2, (z1 + z2) / 2
    for xa, xb in ((x1, xm), (xm, x2)):
        for ya, yb in ((y1, ym), (ym, y2)):
            for za, zb in ((z1, zm), (zm, z2)):
                yield xa, xb, ya, yb, za, zb


@pytest.mark.parametrize("box", [(0.3, 1.7, -0.9, 0.4, 0.0, 1.1), (-3.3, -1.1, 2.2, 5.4, 0.7, 3.9),
                                 (-0.45, 0.55, -0.35, 0.65, 0.0, 0.8)])
def test_subprism_additivity(box):
    """A prism equals the sum of its 8 half-size sub-prisms (the integral is additive)."""
    whole = O.prism_grav(*box)
    parts = sum(O.prism_grav(*b) for b in _split8(*box))
    assert parts == pytest.approx(whole, rel=1e-13, abs=1e-13)
    tw = O.prism_mag_terms(*box)[:5]
    tp = sum(O.prism_mag_terms(*b)[:5] for b in _split8(*box))
    np.testing.assert_allclose(tp, tw, rtol=1e-12, atol=1e-13)


def test_grid_layer_sums_to_one_big_prism():
    """Summing one station's row of G over a padded layer gives the prism of the whole layer."""
    geom = O.Geometry(5, 4, 3, 20.0, 30.0, (0.0, 15.0, 40.0, 70.0), 2, 3, 1, 4, O.GRAVITY)
    k = 2 * geom.sx + 3  # station (i=3, j=2)
    row = O.rows(geom, [k])[0].reshape(geom.nz, geom.ny, geom.nx)
    a = (3 + geom.pxl + 0.5) * geom.dx
    b = (2 + geom.pyl + 0.5) * geom.dy
    for r in range(geom.nz):
        big = GAMMA * O.prism_grav(-a, geom.nx * geom.dx - a, -b, geom.ny * geom.dy - b,
                                   geom.zplanes[r], geom.zplanes[r + 1])
        assert row[r].sum() == pytest.approx(big, rel=1e-12)


# ---------------------------------------------------------------- P4 dipole limit
@pytest.mark.parametrize("incl,decl", [(90.0, 0.0), (50.0, 8.0), (60.0, 0.0), (-35.0, 120.0), (0.0, 45.0)])
def test_dipole_limit_magnetic(incl, decl):
    """A small cube far away gives dT = (F/4pi) kappa V F^.(grad grad 1/r).F^ (induced dipole)."""
    geom = O.Geometry(1, 1, 2, 1.0, 1.0, (0.0, 100.0, 101.0), 0, 300, 0, 300, O.MAGNETIC,
                      incl, decl, 50000.0)
    for p, q in ((120, 40), (7, 150), (0, 0)):
        e = O.entry(geom, 0, 0, p, q, 1)
        x, y, z = p + 0.0, q + 0.0, 100.5
        ref = 50000.0 / (4 * math.pi) * _dipole_integrand(_fhat(incl, decl))(x, y, z)
        assert e == pytest.approx(ref, rel=2e-6, abs=1e-9 * abs(50000.0 / (4 * math.pi) / 100.5 ** 3))


# ---------------------------------------------------------------- P9 quadrature
def test_gravity_entries_match_quadrature():
    """Entries of a padded grid equal gamma * INT z / r^3 dV by Gauss-Legendre quadrature."""
    geom = O.Geometry(4, 3, 3, 20.0, 30.0, (0.0, 15.0, 40.0, 70.0), 1, 2, 2, 1, O.GRAVITY)
    f = lambda X, Y, Z: Z / np.sqrt(X * X + Y * Y + Z * Z) ** 3  # noqa: E731
    rng = np.random.default_rng(7)
    for _ in range(12):
        i, j = int(rng.integers(geom.sx)), int(rng.integers(geom.sy))
        p, q, r = int(rng.integers(geom.nx)), int(rng.integers(geom.ny)), int(rng.integers(1, geom.nz))
        b = _cell_bounds(geom, i, j, p, q, r)
        assert O.entry(geom, i, j, p, q, r) == pytest.approx(GAMMA * _gl3(f, b), rel=1e-11)


@pytest.mark.parametrize("incl,decl", [(50.0, 8.0), (-20.0, 200.0)])
def test_magnetic_entries_match_quadrature(incl, decl):
    """Magnetic entries equal (F/4pi) INT F^.(grad grad 1/r).F^ dV by quadrature, for cells
    at least half a cell from the station (top layer included)."""
    geom = O.Geometry(4, 3, 3, 20.0, 30.0, (0.0, 15.0, 40.0, 70.0), 1, 2, 2, 1, O.MAGNETIC,
                      incl, decl, 48000.0)
    f = _dipole_integrand(_fhat(incl, decl))
    H = 48000.0 / (4 * math.pi)
    rng = np.random.default_rng(11)
    checked = 0
    while checked < 12:
        i, j = int(rng.integers(geom.sx)), int(rng.integers(geom.sy))
        p, q, r = int(rng.integers(geom.nx)), int(rng.integers(geom.ny)), int(rng.integers(geom.nz))
        if r == 0 and p == i + geom.pxl and q == j + geom.pyl:
            continue  # self cell: see test_magnetic_self_cell_is_exterior_limit
        b = _cell_bounds(geom, i, j, p, q, r)
        ref = H * _gl3(f, b, n=32, sub=4)
        assert O.entry(geom, i, j, p, q, r) == pytest.approx(ref, rel=1e-9, abs=1e-12 * H)
        checked += 1


# ---------------------------------------------------------------- far field: rounding of the corner sums
# Far from the station the 8 corner terms of an entry are about r ln r (gravity) or ln r
# (magnetic) while the entry is about V z / r^3: on the 300 x 250 x 60 grid the top-layer
# terms cancel by a factor near 5e11, so an oracle in a 64-bit significand (x87) is off by up
# to 1e-7 there.  These pins hold the oracle to 1e-15 at the farthest offsets of the two largest
# grids, against the same signed corner sum in 50-digit arithmetic and, independently of the
# corner formula, against Gauss-Legendre quadrature of the integrand in 30-digit arithmetic.
FAR_GRAV = O.Geometry.uniform(300, 250, 60, 20.0, 20.0, 20.0, 30, 25)  # 10 % padding per side
FAR_MAG = O.Geometry.uniform(128, 128, 32, 25.0, 25.0, 25.0, 0, 0, O.MAGNETIC, 60.0, 0.0)
FAR_MAG_D = O.Geometry.uniform(64, 64, 16, 25.0, 25.0, 25.0, 3, 3, O.MAGNETIC, 50.0, 8.0)
# (station i, j, cell p, q, r): corners of the grid, the deepest layer, and offsets in between
FAR_G_CASES = [(0, 0, 359, 299, 0), (0, 0, 359, 0, 0), (0, 0, 0, 299, 0), (299, 249, 0, 0, 0),
               (0, 0, 359, 299, 59), (150, 100, 330, 280, 0), (0, 249, 359, 0, 30), (299, 0, 0, 299, 1),
               (0, 0, 30, 299, 0)]
FAR_M_CASES = [(0, 0, 127, 127, 0), (127, 0, 0, 127, 0), (0, 0, 127, 0, 5), (64, 64, 0, 127, 31)]
FAR_MD_CASES = [(0, 0, 69, 69, 0), (63, 0, 0, 69, 0), (0, 63, 69, 0, 15)]


def _corners_mp(geom, i, j, p, q, r):
    """Exact corner offsets of cell (p, q, r) from station (i, j) as mpmath numbers."""
    import mpmath as mp

    x1 = (mp.mpf(p - i - geom.pxl) - mp.mpf(1) / 2) * mp.mpf(geom.dx)
    y1 = (mp.mpf(q - j - geom.pyl) - mp.mpf(1) / 2) * mp.mpf(geom.dy)
    return ((x1, x1 + mp.mpf(geom.dx)), (y1, y1 + mp.mpf(geom.dy)),
            (mp.mpf(geom.zplanes[r]), mp.mpf(geom.zplanes[r + 1])))


def _grav_corner_sum_mp(xs, ys, zs):
    """gamma-free gravity entry as the signed corner sum of Sec. 4.1, plain form."""
    import mpmath as mp

    s = mp.mpf(0)
    for a in range(2):
        for b in range(2):
            for c in range(2):
                x, y, z = xs[a], ys[b], zs[c]
                rho = mp.sqrt(x * x + y * y + z * z)
                t = z * mp.atan(x * y / (z * rho)) if z != 0 else mp.mpf(0)
                f = t - x * mp.log(rho + y) - y * mp.log(rho + x)
                s += f if (a + b + c) % 2 == 1 else -f
    return s


def _mag_corner_sum_mp(xs, ys, zs, coef):
    """Magnetic entry as the five signed corner sums of Sec. 4.2 with the derived coefficients."""
    import mpmath as mp

    L = [mp.mpf(0)] * 5
    for a in range(2):
        for b in range(2):
            for c in range(2):
                x, y, z = xs[a], ys[b], zs[c]
                rho = mp.sqrt(x * x + y * y + z * z)
                mu = 1 if (a + b + c) % 2 == 1 else -1
                terms = (mp.log(rho + x), mp.log(rho + y), mp.log(rho + z),
                         mp.atan(y * z / (x * rho)), mp.atan(x * z / (y * rho)))
                L = [L[k] + mu * terms[k] for k in range(5)]
    return sum(coef[k] * L[k] for k in range(5))


def _mag_coef_mp(geom):
    import mpmath as mp

    I, D = mp.radians(geom.incl_deg), mp.radians(geom.decl_deg)
    l, m, n = mp.cos(I) * mp.cos(D), mp.cos(I) * mp.sin(D), mp.sin(I)
    H = mp.mpf(geom.F_nT) / (4 * mp.pi)
    return [H * 2 * m * n, H * 2 * l * n, H * 2 * l * m, H * (n * n - l * l), H * (n * n - m * m)]


def test_far_field_entries_match_50_digit_corner_sums():
    """The oracle's far-field entries agree with the same corner sums in 50-digit arithmetic."""
    import mpmath as mp

    assert O.significand_bits() == 113
    with mp.workdps(50):
        gamma = mp.mpf("6.67430e-3")
        for c in FAR_G_CASES:
            ref = gamma * _grav_corner_sum_mp(*_corners_mp(FAR_GRAV, *c))
            got = O.entry(FAR_GRAV, *c)
            assert abs(got - ref) <= 1e-15 * abs(ref), (c, got, ref)
        for geom, cases in ((FAR_MAG, FAR_M_CASES), (FAR_MAG_D, FAR_MD_CASES)):
            coef = _mag_coef_mp(geom)
            for c in cases:
                ref = _mag_corner_sum_mp(*_corners_mp(geom, *c), coef)
                got = O.entry(geom, *c)
                assert abs(got - ref) <= 1e-15 * abs(ref), (c, got, ref)


def _gl3_mp(f, bounds, n=6):
    """Tensor Gauss-Legendre integral of f over a box in the current mpmath precision."""
    import mpmath as mp

    X, W = mp.mp.gauss_quadrature(n, "legendre")
    (x1, x2), (y1, y2), (z1, z2) = bounds
    hx, hy, hz = (x2 - x1) / 2, (y2 - y1) / 2, (z2 - z1) / 2
    cx, cy, cz = (x2 + x1) / 2, (y2 + y1) / 2, (z2 + z1) / 2
    tot = mp.mpf(0)
    for a in range(n):
        for b in range(n):
            for c in range(n):
                tot += W[a] * W[b] * W[c] * f(cx + hx * X[a], cy + hy * X[b], cz + hz * X[c])
    return tot * hx * hy * hz


def test_far_field_entries_match_quadrature_of_the_integrand():
    """Independently of the corner formula: far-field entries equal the quadrature of
    gamma z / r^3 (gravity) and of (F/4pi) F^.(grad grad 1/r).F^ (magnetic) to 1e-14; six nodes
    per axis are exact to ~(cell / 2r)^12 there."""
    import mpmath as mp

    with mp.workdps(30):
        gamma = mp.mpf("6.67430e-3")
        grav = lambda x, y, z: z / mp.sqrt(x * x + y * y + z * z) ** 3  # noqa: E731
        for c in FAR_G_CASES[:6]:
            ref = gamma * _gl3_mp(grav, _corners_mp(FAR_GRAV, *c))
            got = O.entry(FAR_GRAV, *c)
            assert abs(got - ref) <= 1e-14 * abs(ref), (c, got, ref)
        for geom, cases in ((FAR_MAG, FAR_M_CASES), (FAR_MAG_D, FAR_MD_CASES)):
            I, D = mp.radians(geom.incl_deg), mp.radians(geom.decl_deg)
            fh = (mp.cos(I) * mp.cos(D), mp.cos(I) * mp.sin(D), mp.sin(I))
            H = mp.mpf(geom.F_nT) / (4 * mp.pi)

            def dip(x, y, z):
                r2 = x * x + y * y + z * z
                s = 3 * (fh[0] * x + fh[1] * y + fh[2] * z) ** 2 - r2 * (fh[0] ** 2 + fh[1] ** 2 + fh[2] ** 2)
                return s / (r2 * r2 * mp.sqrt(r2))

            for c in cases:
                ref = H * _gl3_mp(dip, _corners_mp(geom, *c))
                got = O.entry(geom, *c)
                assert abs(got - ref) <= 1e-14 * abs(ref), (c, got, ref)


# ---------------------------------------------------------------- self cell (P13, R8)
def test_gravity_self_cell_semi_analytic():
    """Station at the centre of the top face of its cell: the z-integral of z/r^3 is
    1/s - 1/sqrt(s^2 + h^2); the singular part integrates to 8 a asinh(1) over the square
    [-a, a]^2 and the smooth part by Gauss-Legendre."""
    a, h = 25.0, 50.0
    geom = O.Geometry(1, 1, 1, 2 * a, 2 * a, (0.0, h), 0, 0, 0, 0, O.GRAVITY)
    x, w = leggauss(64)
    X, Y = np.meshgrid(a * x, a * x, indexing="ij")
    smooth = np.sum(np.outer(w, w) * a * a / np.sqrt(X * X + Y * Y + h * h))
    ref = GAMMA * (8 * a * math.asinh(1.0) - smooth)
    assert O.entry(geom, 0, 0, 0, 0, 0) == pytest.approx(ref, rel=1e-12)


def test_magnetic_self_cell_is_exterior_limit():
    """The magnetic self-cell entry is the limit of the entry for a station raised by delta
    above its cell (Laplace form continuous across the face); off the face all forms agree."""
    for incl, decl in ((50.0, 8.0), (90.0, 0.0), (10.0, -70.0)):
        on = O.Geometry(1, 1, 1, 25.0, 25.0, (0.0, 25.0), 0, 0, 0, 0, O.MAGNETIC, incl, decl)
        e0 = O.entry(on, 0, 0, 0, 0, 0)
        for delta in (1e-3, 1e-5):
            up = O.Geometry(1, 1, 2, 25.0, 25.0, (0.0, delta, delta + 25.0), 0, 0, 0, 0,
                            O.MAGNETIC, incl, decl)
            e1 = O.entry(up, 0, 0, 0, 0, 1)
            assert abs(e1 - e0) <= 10 * delta / 25.0 * abs(e0) + 1e-9


# ---------------------------------------------------------------- P5 Laplace
def test_laplace_off_and_inside_body():
    """T_xx + T_yy + T_zz = -(A_x + A_y + A_z) is 0 off the body and -4 pi inside it."""
    for box in ((0.5, 1.5, -0.5, 0.5, 0.2, 1.2), (-3.0, -1.0, 2.0, 4.0, 1.0, 2.0)):
        t = O.prism_mag_terms(*box)
        assert abs(t[3] + t[4] + t[5]) < 1e-13
    t = O.prism_mag_terms(-0.4, 0.6, -0.7, 0.3, -0.2, 0.9)
    assert t[3] + t[4] + t[5] == pytest.approx(4 * math.pi, rel=1e-13)


# ---------------------------------------------------------------- P6 symmetries
def test_gravity_kernel_even_symmetries():
    """Gravity: k(dx,dy) = k(-dx,dy) = k(dx,-dy), and k(dx,dy) = k(dy,dx) when dx = dy."""
    geom = O.Geometry(1, 1, 2, 20.0, 20.0, (0.0, 20.0, 40.0), 6, 6, 6, 6, O.GRAVITY)
    c = 6  # padded index of the station's own cell
    for dx_, dy_ in ((1, 0), (2, 3), (5, 1), (4, 6)):
        for r in range(2):
            v = O.entry(geom, 0, 0, c + dx_, c + dy_, r)
            for sx_, sy_ in ((-1, 1), (1, -1), (-1, -1)):
                assert O.entry(geom, 0, 0, c + sx_ * dx_, c + sy_ * dy_, r) == pytest.approx(v, rel=1e-14)
            assert O.entry(geom, 0, 0, c + dy_, c + dx_, r) == pytest.approx(v, rel=1e-14)


def test_magnetic_kernel_symmetries():
    """Magnetic: even in both axes at the pole (I = 90), even in dy for D = 0, and in
    general NOT even under (dx,dy) -> (-dx,-dy) -- the non-symmetric BTTB of Sec. 2.2.3."""
    def geom(incl, decl):
        return O.Geometry(1, 1, 2, 20.0, 20.0, (0.0, 20.0, 40.0), 6, 6, 6, 6, O.MAGNETIC, incl, decl)
    c = 6
    pole, d0, gen = geom(90.0, 0.0), geom(60.0, 0.0), geom(50.0, 8.0)
    asym = 0.0
    for dx_, dy_ in ((1, 0), (2, 3), (5, 1), (0, 4)):
        for r in range(2):
            v = O.entry(pole, 0, 0, c + dx_, c + dy_, r)
            for sx_, sy_ in ((-1, 1), (1, -1), (-1, -1)):
                assert O.entry(pole, 0, 0, c + sx_ * dx_, c + sy_ * dy_, r) == pytest.approx(v, rel=1e-12, abs=1e-12)
            v = O.entry(d0, 0, 0, c + dx_, c + dy_, r)
            assert O.entry(d0, 0, 0, c + dx_, c - dy_, r) == pytest.approx(v, rel=1e-12, abs=1e-12)
            a = O.entry(gen, 0, 0, c + dx_, c + dy_, r)
            b = O.entry(gen, 0, 0, c - dx_, c - dy_, r)
            asym = max(asym, abs(a - b) / max(abs(a), abs(b)))
    assert asym > 1e-2


# ---------------------------------------------------------------- P7 Toeplitz invariant
def test_dense_g_is_block_toeplitz_by_layer():
    """Each entry depends only on (p - i, q - j, r) (Sec. 2.1: spatial invariance), exactly."""
    geom = O.Geometry(4, 3, 2, 20.0, 30.0, (0.0, 15.0, 40.0), 2, 1, 1, 3, O.MAGNETIC, 50.0, 8.0)
    G = O.dense(geom).reshape(geom.sy, geom.sx, geom.nz, geom.ny, geom.nx)
    seen = {}
    for j in range(geom.sy):
        for i in range(geom.sx):
            for r in range(geom.nz):
                for q in range(geom.ny):
                    for p in range(geom.nx):
                        key = (p - i, q - j, r)
                        v = G[j, i, r, q, p]
                        if key in seen:
                            assert v == seen[key]
                        else:
                            seen[key] = v
    nx_, ny_ = geom.sx + geom.nx - 1, geom.sy + geom.ny - 1
    assert len(seen) == nx_ * ny_ * geom.nz  # the unique offsets: (s+n-1) per axis, Sec. 3


def test_unpadded_gravity_layer_is_symmetric():
    """Without padding G^(r) is square and symmetric (symBTTB, Sec. 2.2.1)."""
    geom = O.Geometry(5, 4, 2, 20.0, 30.0, (0.0, 15.0, 40.0), 0, 0, 0, 0, O.GRAVITY)
    G = O.dense(geom).reshape(geom.m, geom.nz, geom.m)
    for r in range(geom.nz):
        np.testing.assert_allclose(G[:, r, :], G[:, r, :].T, rtol=1e-14, atol=0)


# ---------------------------------------------------------------- P8 worked examples
def test_worked_example_padded_symmetric_1d():
    """Sec. 2.2.2: s_x = 4, p_xL = 2, p_xR = 1; the real-station rows are toeplitz(c, r) with
    c = (g3, g4, g5, g6), r = (g3, g2, g1, g2, g3, g4, g5), g_k the contribution of block k
    to the first (artificial) station."""
    padded = O.Geometry(4, 1, 1, 20.0, 20.0, (0.0, 20.0), 2, 1, 0, 0, O.GRAVITY)
    full = O.Geometry(7, 1, 1, 20.0, 20.0, (0.0, 20.0), 0, 0, 0, 0, O.GRAVITY)  # stations everywhere
    g = {k: O.entry(full, 0, 0, k - 1, 0, 0) for k in range(1, 8)}
    G = O.dense(padded)
    expect = np.array([[g[3], g[2], g[1], g[2], g[3], g[4], g[5]],
                       [g[4], g[3], g[2], g[1], g[2], g[3], g[4]],
                       [g[5], g[4], g[3], g[2], g[1], g[2], g[3]],
                       [g[6], g[5], g[4], g[3], g[2], g[1], g[2]]])
    np.testing.assert_allclose(G, expect, rtol=1e-14)
    np.testing.assert_array_equal(G, O.dense(full)[2:6])  # rows of the real stations


def test_worked_example_padded_nonsymmetric_1d():
    """Sec. 2.2.4: same sizes, non-symmetric kernel; rows are toeplitz(c, r) with
    c = (gam3, gam4, gam5, gam6), r = (gam3, gam2, g1, g2, g3, g4, g5), where g_k is block k
    seen from station 1 and gam_k is block 1 seen from station k."""
    kw = dict(kind=O.MAGNETIC, incl_deg=50.0, decl_deg=8.0)
    padded = O.Geometry(4, 1, 1, 20.0, 20.0, (0.0, 20.0), 2, 1, 0, 0, **kw)
    full = O.Geometry(7, 1, 1, 20.0, 20.0, (0.0, 20.0), 0, 0, 0, 0, **kw)
    g = {k: O.entry(full, 0, 0, k - 1, 0, 0) for k in range(1, 8)}
    gam = {k: O.entry(full, k - 1, 0, 0, 0, 0) for k in range(1, 8)}
    G = O.dense(padded)
    expect = np.array([[gam[3], gam[2], g[1], g[2], g[3], g[4], g[5]],
                       [gam[4], gam[3], gam[2], g[1], g[2], g[3], g[4]],
                       [gam[5], gam[4], gam[3], gam[2], g[1], g[2], g[3]],
                       [gam[6], gam[5], gam[4], gam[3], gam[2], g[1], g[2]]])
    np.testing.assert_array_equal(G, expect)
    assert abs(g[2] - gam[2]) > 1e-3 * abs(g[2])  # genuinely non-symmetric


# ---------------------------------------------------------------- P10 linearity / adjoint
def test_forward_transpose_dense_consistency():
    """forward == dense G @ m, transpose == dense G^T @ d, <Gm, d> = <m, G^T d>."""
    geom = O.Geometry(5, 3, 2, 20.0, 30.0, (0.0, 15.0, 40.0), 1, 2, 2, 0, O.MAGNETIC, 50.0, 8.0)
    rng = np.random.default_rng(3)
    m, d = rng.standard_normal(geom.n), rng.standard_normal(geom.m)
    G = O.dense(geom)
    Gm = O.forward(geom, m).ravel()
    Gtd = O.transpose(geom, d).ravel()
    assert rel_err(Gm, G @ m) < 1e-14
    assert rel_err(Gtd, G.T @ d) < 1e-14
    assert float(Gm @ d) == pytest.approx(float(m @ Gtd), rel=1e-13)
    m2 = rng.standard_normal(geom.n)
    assert rel_err(O.forward(geom, 2.0 * m - 3.0 * m2).ravel(), 2.0 * Gm - 3.0 * O.forward(geom, m2).ravel()) < 1e-14


def test_sampled_rows_and_cells_match_full():
    geom = O.Geometry(6, 5, 3, 20.0, 30.0, (0.0, 15.0, 40.0, 70.0), 1, 2, 0, 1, O.GRAVITY)
    rng = np.random.default_rng(5)
    m, d = rng.standard_normal(geom.n), rng.standard_normal(geom.m)
    full_f = O.forward(geom, m).ravel()
    full_t = O.transpose(geom, d).ravel()
    st = np.array([0, 7, geom.m - 1])
    cl = np.array([0, 11, geom.n - 1])
    np.testing.assert_array_equal(O.forward(geom, m, st), full_f[st])
    np.testing.assert_array_equal(O.transpose(geom, d, cl), full_t[cl])


# ---------------------------------------------------------------- Table 1
def _five_sig(v):
    e = int(math.floor(math.log10(v))) - 4
    return round(v / 10 ** e) * 10 ** e if e > 0 else v


def test_table1_sizes_reproduce_with_per_side_padding():
    """Table 1: m = s_x s_y, n(0 %) = s_x s_y n_z and n(5 %) with round-half-up(0.05 s) padding
    cells on EACH side; the printed n values of problems 9, 11 and 12 are 5-significant-digit
    roundings (e.g. 662450 is not even divisible by n_z = 18)."""
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "table1_sizes.txt")
    rows = [list(map(int, ln.split())) for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 12
    for k, sx, sy, nz, m, n0, n5 in rows:
        assert (sx, sy, nz) == (25 * k, 15 * k, 2 * k)
        px, py = math.floor(0.05 * sx + 0.5), math.floor(0.05 * sy + 0.5)
        geom = O.Geometry.uniform(sx, sy, nz, 1.0, 1.0, 1.0, px, py)
        assert geom.m == m
        assert sx * sy * nz == n0
        assert _five_sig(geom.n) == n5


def test_bench_table1_sweep_uses_the_table1_geometries():
    """bench.py --table1 builds exactly the sizes of Table 1 (same fixture, same padding rule)."""
    import os
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    path = os.path.join(os.path.dirname(__file__), "golden", "table1_sizes.txt")
    rows = {r[0]: r for r in (list(map(int, ln.split())) for ln in open(path) if ln.strip() and not ln.startswith("#"))}
    seen = set()
    for k, pad, w in bench.table1_workloads(range(1, 13)):
        _, sx, sy, nz, m, n0, n5 = rows[k]
        assert (w.sx, w.sy, w.nz, w.m) == (sx, sy, nz, m)
        assert (w.n if pad == 0 else _five_sig(w.n)) == (n0 if pad == 0 else n5)
        seen.add((k, pad))
    assert len(seen) == 24


def test_scattered_entries_match_dense_rows():
    """entries() (the timing sample unit) returns exactly the dense matrix's entries."""
    geom = O.Geometry.uniform(5, 4, 3, 10.0, 12.0, 8.0, 1, 2, O.MAGNETIC, 60.0, 15.0)
    G = O.dense(geom)
    rng = np.random.default_rng(5)
    st = rng.integers(0, geom.m, 200)
    ce = rng.integers(0, geom.n, 200)
    assert np.array_equal(O.entries(geom, st, ce), G[st, ce])
