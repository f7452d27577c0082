/*
 * gm_oracle.c -- CPU oracle for the gravity / magnetic prism forward operator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg use it.  It shares no code, header, table or helper with the
 * CUDA path.
 *
 * What it computes is the plain definition of the sensitivity matrix G of
 * Hogue, Renaut & Vatankhah (arXiv 1912.06976), Sec. 2 (Eqs. stationsij,
 * prismspqr, Gslice, htilde): one entry per (station, prism) pair, each entry
 * the closed-form prism integral of Sec. 4, evaluated corner by corner, and
 * then d = G m and m' = G^T d by direct summation.  There is no Toeplitz,
 * circulant or FFT code here, no corner-grid reuse and no reordering: every
 * entry is evaluated from its own 8 corners.
 *
 * Arithmetic is IEEE binary128 (113-bit significand): long double on
 * aarch64, __float128 with libquadmath on x86-64 (where long double is only
 * the 64-bit-significand x87 format); the build refuses any other format.
 * Far from the station the 8 corner terms of an entry cancel: their size is
 * about r ln r while the entry is about dx dy dz z / r^3, a ratio near 4e11
 * for a 20 m top-layer cell 7.8 km away.  In binary128 (eps = 1.9e-34) that
 * cancellation leaves about 1e-22 relative error, far below the 1e-12 gate
 * the FP64 GPU path is held to; the x87 format (eps = 1.1e-19) would leave
 * up to 1e-7 at such entries, which is why it is not used.
 *
 * Geometry (0-based; Sec. 2.1.1-2.1.2, Eq. PaddedDistances and the notation
 * table of App. A):
 *   stations (i, j), 0 <= i < sx, 0 <= j < sy, at depth 0, at the centres of
 *     the top faces of the unpadded cells:  a_i = (i + pxl + 1/2) dx,
 *     b_j = (j + pyl + 1/2) dy;
 *   cells (p, q, r), 0 <= p < nx = sx + pxl + pxr, 0 <= q < ny, 0 <= r < nz,
 *     spanning [p dx, (p+1) dx] x [q dy, (q+1) dy] x [z_r, z_{r+1}];
 *   z positive down; the stations are at depth 0 and the layer boundaries
 *   z_0 < z_1 < ... < z_nz (z_0 >= 0) are given (z_blocks of App. A).
 *   Row index of G:    k = j*sx + i        (x fastest, Eq. htilde)
 *   Column index of G: l = (r*ny + q)*nx + p
 *
 * Gravity entry (Sec. 4.1, the Boulanger-Chouteau / Haaz prism formula):
 *   G = gamma * SUM_{corners} mu * [ z atan(x y / (z rho)) - x ln(rho + y)
 *                                    - y ln(rho + x) ],
 *   rho = sqrt(x^2 + y^2 + z^2), (x, y, z) the corner relative to the
 *   station, mu = +1 on an even number of lower limits, -1 on an odd number
 *   (the (-1)^i (-1)^j (-1)^k of Sec. 4.1).  gamma = 6.67430e-3 turns
 *   g/cm^3 and metres into mGal.  The z*atan term is 0 at z = 0.
 *
 * Magnetic entry (Sec. 4.2, Eq. magnetickernel; induced magnetisation only):
 *   G = (F / 4 pi) * [ (n^2 - l^2) A_x + (n^2 - m^2) A_y
 *                      + 2 l m L_z + 2 l n L_y + 2 m n L_x ]
 *   with L_x = S[ln(rho + x)], L_y = S[ln(rho + y)], L_z = S[ln(rho + z)],
 *        A_x = S[atan(y z / (x rho))], A_y = S[atan(x z / (y rho))],
 *   S[.] the same signed 8-corner sum, x = North, y = East, z = Down,
 *   (l, m, n) = (cos I cos D, cos I sin D, sin I) and F in nT.  The paper
 *   does not print its constants G_1..G_5; these follow from
 *   dT = (F/4pi) kappa SUM_ab Fhat_a Fhat_b d_a d_b INT 1/r dV with
 *   T_xx = -A_x, T_yy = -A_y, T_xy = L_z, T_xz = L_y, T_yz = L_x and T_zz
 *   eliminated through Laplace's equation (T_zz = A_x + A_y), which is also
 *   the exterior limit for a station on the top face of its own cell.  The
 *   pins in tests/test_oracle_pins.py (dipole limit, Gauss-Legendre
 *   quadrature, Laplace) fix these constants and signs.
 *
 * Stable forms: for x < 0, rho + x = (y^2 + z^2) / (rho - x) (likewise for y
 * and z), which avoids the cancellation of rho + x when |x| ~ rho.
 */
#include <float.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#if LDBL_MANT_DIG == 113
typedef long double ld; /* IEEE binary128 */
#define LDC(x) x##L
#define ld_log logl
#define ld_atan atanl
#define ld_sqrt sqrtl
#define ld_cos cosl
#define ld_sin sinl
#define GMO_MANT_DIG LDBL_MANT_DIG
#elif defined(__SIZEOF_FLOAT128__)
#include <quadmath.h>
typedef __float128 ld; /* IEEE binary128 in software */
#define LDC(x) x##Q
#define ld_log logq
#define ld_atan atanq
#define ld_sqrt sqrtq
#define ld_cos cosq
#define ld_sin sinq
#define GMO_MANT_DIG FLT128_MANT_DIG
#else
#error "the oracle needs IEEE binary128 arithmetic (long double on aarch64 or __float128)"
#endif

#define GMO_GRAVITY 0
#define GMO_MAGNETIC 1

/* Geometry record shared with the Python wrapper (oracle/oracle.py). */
typedef struct {
    int sx, sy, nz;
    int pxl, pxr, pyl, pyr;
    double dx, dy;
    const double *zplanes; /* nz + 1 increasing layer boundaries (m), zplanes[0] >= 0 */
    int kind;              /* GMO_GRAVITY or GMO_MAGNETIC */
    double incl_deg, decl_deg, F_nT;
} gmo_geom;

static const ld GMO_GAMMA = LDC(6.67430e-3); /* mGal per (g/cm^3 * m) */
static const ld GMO_PI = LDC(3.14159265358979323846264338327950288);

/* ln(rho + a) where rho = sqrt(a^2 + b2), b2 = sum of the squares of the
 * two other coordinates.  For a < 0 the sum is rewritten as b2 / (rho - a). */
static ld ln_rho_plus(ld a, ld b2, ld rho) {
    if (a >= LDC(0.0)) return ld_log(rho + a);
    return ld_log(b2 / (rho - a));
}

/* The gravity corner function of Sec. 4.1 at one corner. */
static ld grav_corner(ld x, ld y, ld z) {
    ld x2 = x * x, y2 = y * y, z2 = z * z;
    ld rho = ld_sqrt(x2 + y2 + z2);
    ld t = LDC(0.0);
    if (z != LDC(0.0)) t = z * ld_atan((x * y) / (z * rho));
    return t - x * ln_rho_plus(y, x2 + z2, rho) - y * ln_rho_plus(x, y2 + z2, rho);
}

/* Signed 8-corner sum of the gravity corner function over the prism
 * [x1,x2] x [y1,y2] x [z1,z2], relative to a station at the origin; upper
 * limits carry +, so a prism below the station gives a positive value. */
static ld grav_prism_ld(ld x1, ld x2, ld y1, ld y2, ld z1, ld z2) {
    const ld xs[2] = {x1, x2}, ys[2] = {y1, y2}, zs[2] = {z1, z2};
    ld s = LDC(0.0);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c) {
                int lower = (a == 0) + (b == 0) + (c == 0);
                ld mu = (lower & 1) ? -LDC(1.0) : LDC(1.0);
                s += mu * grav_corner(xs[a], ys[b], zs[c]);
            }
    return s;
}

double gmo_prism_grav(double x1, double x2, double y1, double y2, double z1, double z2) {
    return (double)grav_prism_ld(x1, x2, y1, y2, z1, z2);
}

/* The six magnetic corner sums of the prism: out = {L_x, L_y, L_z, A_x, A_y,
 * A_z} with A_z = S[atan(x y / (z rho))] (A_z is not used by the entry; it
 * lets the tests check Laplace's equation). */
static void mag_terms_ld(ld x1, ld x2, ld y1, ld y2, ld z1, ld z2, ld out[6]) {
    const ld xs[2] = {x1, x2}, ys[2] = {y1, y2}, zs[2] = {z1, z2};
    ld Lx = 0, Ly = 0, Lz = 0, Ax = 0, Ay = 0, Az = 0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c) {
                int lower = (a == 0) + (b == 0) + (c == 0);
                ld mu = (lower & 1) ? -LDC(1.0) : LDC(1.0);
                ld x = xs[a], y = ys[b], z = zs[c];
                ld x2 = x * x, y2 = y * y, z2 = z * z;
                ld rho = ld_sqrt(x2 + y2 + z2);
                Lx += mu * ln_rho_plus(x, y2 + z2, rho);
                Ly += mu * ln_rho_plus(y, x2 + z2, rho);
                Lz += mu * ln_rho_plus(z, x2 + y2, rho);
                Ax += mu * ld_atan((y * z) / (x * rho));
                Ay += mu * ld_atan((x * z) / (y * rho));
                if (z != LDC(0.0)) Az += mu * ld_atan((x * y) / (z * rho));
                else Az += mu * (((x * y) > LDC(0.0)) ? GMO_PI / 2 : -GMO_PI / 2);
            }
    out[0] = Lx; out[1] = Ly; out[2] = Lz; out[3] = Ax; out[4] = Ay; out[5] = Az;
}

void gmo_prism_mag_terms(double x1, double x2, double y1, double y2, double z1, double z2,
                         double out[6]) {
    ld t[6];
    mag_terms_ld(x1, x2, y1, y2, z1, z2, t);
    for (int k = 0; k < 6; ++k) out[k] = (double)t[k];
}

/* The five coefficients of Eq. magnetickernel (already multiplied by F/4pi),
 * in the order of the terms {L_x, L_y, L_z, A_x, A_y}. */
static void mag_coeffs(const gmo_geom *g, ld c[5]) {
    ld I = (ld)g->incl_deg * GMO_PI / LDC(180.0), D = (ld)g->decl_deg * GMO_PI / LDC(180.0);
    ld l = ld_cos(I) * ld_cos(D), m = ld_cos(I) * ld_sin(D), n = ld_sin(I);
    ld H = (ld)g->F_nT / (LDC(4.0) * GMO_PI);
    c[0] = H * LDC(2.0) * m * n;     /* L_x: T_yz */
    c[1] = H * LDC(2.0) * l * n;     /* L_y: T_xz */
    c[2] = H * LDC(2.0) * l * m;     /* L_z: T_xy */
    c[3] = H * (n * n - l * l);  /* A_x: -T_xx + T_zz share */
    c[4] = H * (n * n - m * m);  /* A_y: -T_yy + T_zz share */
}

void gmo_mag_coeffs(const gmo_geom *g, double out[5]) {
    ld c[5];
    mag_coeffs(g, c);
    for (int k = 0; k < 5; ++k) out[k] = (double)c[k];
}

/* Entry G[k, l] with k = j*sx + i and l = (r*ny + q)*nx + p. */
static ld entry_ld(const gmo_geom *g, const ld mc[5], int i, int j, int p, int q, int r) {
    ld x1 = ((ld)(p - i - g->pxl) - LDC(0.5)) * (ld)g->dx;
    ld x2 = x1 + (ld)g->dx;
    ld y1 = ((ld)(q - j - g->pyl) - LDC(0.5)) * (ld)g->dy;
    ld y2 = y1 + (ld)g->dy;
    ld z1 = (ld)g->zplanes[r];
    ld z2 = (ld)g->zplanes[r + 1];
    if (g->kind == GMO_GRAVITY) return GMO_GAMMA * grav_prism_ld(x1, x2, y1, y2, z1, z2);
    ld t[6];
    mag_terms_ld(x1, x2, y1, y2, z1, z2, t);
    return mc[0] * t[0] + mc[1] * t[1] + mc[2] * t[2] + mc[3] * t[3] + mc[4] * t[4];
}

double gmo_entry(const gmo_geom *g, int i, int j, int p, int q, int r) {
    ld mc[5] = {0, 0, 0, 0, 0};
    if (g->kind == GMO_MAGNETIC) mag_coeffs(g, mc);
    return (double)entry_ld(g, mc, i, j, p, q, r);
}

static int gmo_nx(const gmo_geom *g) { return g->sx + g->pxl + g->pxr; }
static int gmo_ny(const gmo_geom *g) { return g->sy + g->pyl + g->pyr; }

/* Dense row block: G[k, :] for each station k listed in rows[0..nrows). */
void gmo_rows(const gmo_geom *g, const int64_t *rows, int64_t nrows, double *out) {
    const int nx = gmo_nx(g), ny = gmo_ny(g);
    const int64_t n = (int64_t)nx * ny * g->nz;
    ld mc[5] = {0, 0, 0, 0, 0};
    if (g->kind == GMO_MAGNETIC) mag_coeffs(g, mc);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < nrows; ++t) {
        int i = (int)(rows[t] % g->sx), j = (int)(rows[t] / g->sx);
        for (int r = 0; r < g->nz; ++r)
            for (int q = 0; q < ny; ++q)
                for (int p = 0; p < nx; ++p)
                    out[t * n + ((int64_t)r * ny + q) * nx + p] = (double)entry_ld(g, mc, i, j, p, q, r);
    }
}

/* Scattered entries: out[t] = G[stations[t], cells[t]] for t < n (stations k = j*sx + i, cells
 * l = (r*ny + q)*nx + p); the unit of work of the oracle's products, for timing samples. */
void gmo_entries(const gmo_geom *g, const int64_t *stations, const int64_t *cells, int64_t n, double *out) {
    const int nx = gmo_nx(g), ny = gmo_ny(g);
    ld mc[5] = {0, 0, 0, 0, 0};
    if (g->kind == GMO_MAGNETIC) mag_coeffs(g, mc);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < n; ++t) {
        const int i = (int)(stations[t] % g->sx), j = (int)(stations[t] / g->sx);
        const int64_t l = cells[t];
        const int p = (int)(l % nx), q = (int)((l / nx) % ny), r = (int)(l / ((int64_t)nx * ny));
        out[t] = (double)entry_ld(g, mc, i, j, p, q, r);
    }
}

/* d[k] = SUM_l G[k, l] m[l] for the stations listed in rows (all stations
 * when rows == NULL, in which case nrows must be sx*sy).  Sums in binary128. */
void gmo_forward(const gmo_geom *g, const double *m, const int64_t *rows, int64_t nrows,
                 double *d) {
    const int nx = gmo_nx(g), ny = gmo_ny(g);
    ld mc[5] = {0, 0, 0, 0, 0};
    if (g->kind == GMO_MAGNETIC) mag_coeffs(g, mc);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < nrows; ++t) {
        int64_t k = rows ? rows[t] : t;
        int i = (int)(k % g->sx), j = (int)(k / g->sx);
        ld acc = LDC(0.0);
        for (int r = 0; r < g->nz; ++r)
            for (int q = 0; q < ny; ++q)
                for (int p = 0; p < nx; ++p)
                    acc += entry_ld(g, mc, i, j, p, q, r) * (ld)m[((int64_t)r * ny + q) * nx + p];
        d[t] = (double)acc;
    }
}

/* m'[l] = SUM_k G[k, l] d[k] for the cells listed in cols (all cells when
 * cols == NULL, in which case ncols must be nx*ny*nz). */
void gmo_transpose(const gmo_geom *g, const double *d, const int64_t *cols, int64_t ncols,
                   double *mout) {
    const int nx = gmo_nx(g), ny = gmo_ny(g);
    ld mc[5] = {0, 0, 0, 0, 0};
    if (g->kind == GMO_MAGNETIC) mag_coeffs(g, mc);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < ncols; ++t) {
        int64_t l = cols ? cols[t] : t;
        int p = (int)(l % nx);
        int q = (int)((l / nx) % ny);
        int r = (int)(l / ((int64_t)nx * ny));
        ld acc = LDC(0.0);
        for (int j = 0; j < g->sy; ++j)
            for (int i = 0; i < g->sx; ++i)
                acc += entry_ld(g, mc, i, j, p, q, r) * (ld)d[(int64_t)j * g->sx + i];
        mout[t] = (double)acc;
    }
}

/* Number of threads the parallel loops above run on (1 without OpenMP). */
int gmo_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void gmo_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Significand bits of the arithmetic type (113 for binary128), so tests and
 * stored samples can state which format ran. */
int gmo_mant_dig(void) { return GMO_MANT_DIG; }
