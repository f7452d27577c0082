// setup.cu -- set-up of a plan: prism entries in FP64, circulant generators, spectra.
//
// Algorithms symBTTBFFT / BTTBFFT (App. B) with the gravity and magnetic
// entry functions of Sec. 4, re-organised for the device:
//
//  K1 k_corner_columns: for every layer r and every corner (x_a, y_b) of the
//     offset grid (Eq. PaddedDistances: x_a = (a + dmin_x - 1/2) dx, a <= N_x),
//     Q_r(x, y) = Phi(x, y, z_{r+1}) - Phi(x, y, z_r), the depth difference of
//     the corner function.  As in the paper's simplification (Sec. 4.1, Eq.
//     simplifiedCMX: ln((x+R1)/(x+R2)) instead of two logs), the difference is
//     taken inside the logarithms and arctangents, here in forms with no
//     cancellation (log1p of the relative increment, atan of the tangent of the
//     angle difference), which keeps far-field entries accurate in FP64.
//  K2 k_generator: the 4-point difference over the corners of each cell offset
//     gives the entry k_r(delta) (Sec. 4.1: g = CM(1:,1:) - CM(1:,2:) - ...);
//     entry k_r(delta) with delta = -u - pxl is written at generator position
//     (u mod N'_x, v mod N'_y) for u in [-(nx-1), sx-1] (Eqs. Tcircpadded,
//     Tcircpaddedgeneral), zeros elsewhere.  That difference cancels by about
//     (r / cell)^2 at distance r (~1e-13 relative error in FP64 for the far and
//     deep cells of a 300 x 250 x 60 grid), so cells whose horizontal gap to the
//     station is at least 2.5 cell widths (2.5 layer thicknesses too, for the
//     magnetic kernel) take instead the defining integral by Gauss-Legendre
//     quadrature, which has no cancellation there: gravity, gamma times the
//     (x, y) face integral of the depth integral of z / r^3, 1/r1 - 1/r2 =
//     (z2^2 - z1^2) / (r1 r2 (r1 + r2)), with 8 x 8 nodes; magnetic, F / 4pi
//     times the volume integral of Fhat . (grad grad 1/r) . Fhat =
//     (3 (Fhat . r)^2 - r^2) / r^5 with 8 x 8 x 8 nodes.  The integrands'
//     nearest singularity, at the station, is at least five half cell widths
//     away, which bounds the quadrature error near 1e-16.
//  K3 2-D FFT of each generator in FP64 (rows, then columns), then rounding
//     to the apply precision.
#include <cstring>
#include <cuda_runtime.h>

#include <cmath>

#include "gm_kernels.cuh"
#include "gm_plan.h"

namespace gm {

// ln(rho2 + a) - ln(rho1 + a) with rho_k = sqrt(a^2 + b2 + z_k^2), z2 > z1 >= 0.
__device__ __forceinline__ double dlog_rho_plus(double a, double b2, double z1, double z2, double r1,
                                                double r2) {
    const double dz2 = (z2 - z1) * (z2 + z1);
    const double drho = dz2 / (r1 + r2);
    if (a >= 0.0) return log1p(drho / (a + r1));
    // rho_k + a = (b2 + z_k^2) / (rho_k - a)
    return log1p(dz2 / (b2 + z1 * z1)) - log1p(drho / (r1 - a));
}

// Gravity: Phi = z atan(x y / (z rho)) - x ln(rho + y) - y ln(rho + x) (Sec. 4.1).
__device__ double q_gravity(double x, double y, double z1, double z2) {
    const double R2 = x * x + y * y;
    const double r1 = sqrt(R2 + z1 * z1), r2 = sqrt(R2 + z2 * z2);
    double at;
    if (z1 == 0.0) {
        at = z2 * atan(x * y / (z2 * r2));
    } else {
        // atan(c2) - atan(c1) = atan((c2 - c1) / (1 + c1 c2)), c_k = x y / (z_k rho_k) of one sign
        const double num = -x * y * (z2 - z1) * (z2 + z1) * (R2 + z1 * z1 + z2 * z2);
        const double den = (z2 * r2 + z1 * r1) * (z1 * z2 * r1 * r2 + x * x * y * y);
        at = z2 * atan(num / den) + (z2 - z1) * atan(x * y / (z1 * r1));
    }
    return at - x * dlog_rho_plus(y, x * x, z1, z2, r1, r2) - y * dlog_rho_plus(x, y * y, z1, z2, r1, r2);
}

// Magnetic (Sec. 4.2, Eq. magnetickernel): c . {dLx, dLy, dLz, dAx, dAy}.
__device__ double q_magnetic(double x, double y, double z1, double z2, const double c[5]) {
    const double R2 = x * x + y * y;
    const double r1 = sqrt(R2 + z1 * z1), r2 = sqrt(R2 + z2 * z2);
    const double dz2 = (z2 - z1) * (z2 + z1);
    const double Lx = dlog_rho_plus(x, y * y, z1, z2, r1, r2);
    const double Ly = dlog_rho_plus(y, x * x, z1, z2, r1, r2);
    const double Lz = log1p((z2 - z1 + dz2 / (r1 + r2)) / (z1 + r1));
    // atan(a2) - atan(a1) with a_k = y z_k / (x rho_k) (one sign): atan((a2-a1)/(1+a1 a2))
    const double k = x * y * R2 * dz2 / (z2 * r1 + z1 * r2);
    const double Ax = atan(k / (x * x * r1 * r2 + y * y * z1 * z2));
    const double Ay = atan(k / (y * y * r1 * r2 + x * x * z1 * z2));
    return c[0] * Lx + c[1] * Ly + c[2] * Lz + c[3] * Ax + c[4] * Ay;
}

struct CornerArgs {
    int ncx, ncy, nz;     // corners per axis (N_x + 1, N_y + 1), layers
    double x0, y0;        // coordinate of corner 0 (metres)
    double dx, dy;
    const double *z;      // nz + 1 depths (device)
    int kind;
    double c[5];          // magnetic coefficients, or {gamma} for gravity
};

// K1: Q[r][b][a] for a < ncx, b < ncy, r < nz.
__global__ void k_corner_columns(double *__restrict__ Q, CornerArgs a) {
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iy = blockIdx.y;
    const int r = blockIdx.z;
    if (ix >= a.ncx) return;
    const double x = a.x0 + ix * a.dx;
    const double y = a.y0 + iy * a.dy;
    const double z1 = a.z[r], z2 = a.z[r + 1];
    double q = (a.kind == GM_GRAVITY) ? a.c[0] * q_gravity(x, y, z1, z2) : q_magnetic(x, y, z1, z2, a.c);
    Q[((size_t)r * a.ncy + iy) * a.ncx + ix] = q;
}

// Far-field quadrature of the entries (K2): quad = 1 gravity (face integral), 2 magnetic (volume
// integral), 0 none; cells whose horizontal gap to the station is at least gap_cells cell widths
// (and, for the magnetic kernel, as many layer thicknesses) use Gauss-Legendre rules on [-1, 1];
// the others keep the 4-point corner difference.  The rule's error falls geometrically with the
// number of nodes and the gap; measured against the binary128 oracle on the 300 x 250 x 60 grid
// (worst relative error in the top layer), 8 nodes per axis reach rounding level (3e-16) from a
// 2.5-width gap, 6 nodes from 9.5, 5 from 19.5 and 4 from 39.5, which set the switch points.
constexpr int kFarNodes = 8;
constexpr double kPiSetup = 3.14159265358979323846264338327950288;
struct GaussRule {
    double x[kFarNodes], w[kFarNodes];
};
struct FarField {
    int quad;
    double gap_cells;
    double x0, y0, dx, dy, gamma;  // corner 0 of the offset grid, cell sizes, gravity constant
    double H, l, m, n;             // magnetic: F / 4pi and the direction cosines of Fhat
    const double *z;
    GaussRule g8, g6, g5, g4;      // 8-, 6-, 5- and 4-point rules
};

// (F / 4pi) * integral over the cell of (3 (Fhat . r)^2 - r^2) / r^5 (Sec. 4.2's entry, the
// induced dipole field along Fhat)
template <int NQ>
__device__ double mag_volume_quadrature(const FarField &f, const GaussRule &q, double xl, double yl, double z1,
                                        double z2) {
    const double hx = 0.5 * f.dx, hy = 0.5 * f.dy, hz = 0.5 * (z2 - z1);
    const double cx = xl + hx, cy = yl + hy, cz = z1 + hz;
    double s = 0.0;
    for (int i = 0; i < NQ; ++i) {
        const double x = cx + hx * q.x[i];
        for (int j = 0; j < NQ; ++j) {
            const double y = cy + hy * q.x[j];
            const double u = f.l * x + f.m * y, rho2 = x * x + y * y;
            double sk = 0.0;
#pragma unroll
            for (int k = 0; k < NQ; ++k) {
                const double z = cz + hz * q.x[k];
                const double r2 = rho2 + z * z, t = u + f.n * z;
                sk += q.w[k] * (3.0 * t * t - r2) / (r2 * r2 * sqrt(r2));
            }
            s += q.w[i] * q.w[j] * sk;
        }
    }
    return f.H * s * hx * hy * hz;
}

// gamma * integral over [xl, xl + dx] x [yl, yl + dy] of (z2^2 - z1^2) / (r1 r2 (r1 + r2)),
// r_k = sqrt(x^2 + y^2 + z_k^2): the depth integral of z / r^3 over [z1, z2] (Sec. 4.1's entry)
template <int NQ>
__device__ double grav_face_quadrature(const FarField &f, const GaussRule &q, double xl, double yl, double z1,
                                       double z2) {
    const double hx = 0.5 * f.dx, hy = 0.5 * f.dy, cx = xl + hx, cy = yl + hy;
    const double dz2 = (z2 - z1) * (z2 + z1), a1 = z1 * z1, a2 = z2 * z2;
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        const double x = cx + hx * q.x[i], x2 = x * x;
        double si = 0.0;
#pragma unroll
        for (int j = 0; j < NQ; ++j) {
            const double y = cy + hy * q.x[j], R2 = x2 + y * y;
            const double r1 = sqrt(R2 + a1), r2 = sqrt(R2 + a2);
            si += q.w[j] / (r1 * r2 * (r1 + r2));
        }
        s += q.w[i] * si;
    }
    return f.gamma * dz2 * s * hx * hy;
}

// the entry of a far cell with the rule its gap needs (gap_w: the gap in units of the largest
// cell width, or layer thickness for the magnetic kernel)
__device__ double far_entry(const FarField &f, double gap_w, double xl, double yl, double z1, double z2) {
    if (f.quad == 1) {
        if (gap_w >= 39.5) return grav_face_quadrature<4>(f, f.g4, xl, yl, z1, z2);
        if (gap_w >= 19.5) return grav_face_quadrature<5>(f, f.g5, xl, yl, z1, z2);
        if (gap_w >= 9.5) return grav_face_quadrature<6>(f, f.g6, xl, yl, z1, z2);
        return grav_face_quadrature<8>(f, f.g8, xl, yl, z1, z2);
    }
    if (gap_w >= 39.5) return mag_volume_quadrature<4>(f, f.g4, xl, yl, z1, z2);
    if (gap_w >= 19.5) return mag_volume_quadrature<5>(f, f.g5, xl, yl, z1, z2);
    if (gap_w >= 9.5) return mag_volume_quadrature<6>(f, f.g6, xl, yl, z1, z2);
    return mag_volume_quadrature<8>(f, f.g8, xl, yl, z1, z2);
}

// K2: generator T[r][vy][ux] (real, FP64) from the corner columns, or by quadrature far out.
__global__ void k_generator(const double *__restrict__ Q, double *__restrict__ T, Geo g, int ncx, int ncy,
                            FarField f) {
    const int ux = blockIdx.x * blockDim.x + threadIdx.x;
    const int vy = blockIdx.y;
    const int r = blockIdx.z;
    if (ux >= g.NPx) return;
    const int u = (ux < g.sx) ? ux : ux - g.NPx;
    const int v = (vy < g.sy) ? vy : vy - g.NPy;
    double t = 0.0;
    if (u >= -(g.nx - 1) && v >= -(g.ny - 1)) {
        // corner index of the lower x edge of offset delta_x = -u - pxl:  sx - 1 - u
        const int xi = g.sx - 1 - u, yi = g.sy - 1 - v;
        const int ddx = -u - g.pxl, ddy = -v - g.pyl;  // cell offset from the station, in cells
        // horizontal gap between the station and the cell (a lower bound of their distance)
        const double gap = fmax((abs(ddx) - 0.5) * f.dx, (abs(ddy) - 0.5) * f.dy);
        const double z1 = f.z[r], z2 = f.z[r + 1];
        double scale = fmax(f.dx, f.dy);
        if (f.quad == 2) scale = fmax(scale, z2 - z1);
        if (f.quad && gap >= f.gap_cells * scale) {
            t = far_entry(f, gap / scale, f.x0 + xi * f.dx, f.y0 + yi * f.dy, z1, z2);
        } else {
            const double *Qr = Q + (size_t)r * ncy * ncx;
            t = Qr[(size_t)(yi + 1) * ncx + xi + 1] - Qr[(size_t)(yi + 1) * ncx + xi] -
                Qr[(size_t)yi * ncx + xi + 1] + Qr[(size_t)yi * ncx + xi];
        }
    }
    T[((size_t)r * g.NPy + vy) * g.NPx + ux] = t;
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton's iteration on the Legendre polynomial
// P_n from the Chebyshev-like first guesses, in long double), rounded to double.
static void gauss_legendre(int n, double *x, double *w) {
    const long double pi = 3.14159265358979323846264338327950288L;
    for (int i = 0; i < n; ++i) {
        long double t = cosl(pi * ((long double)i + 0.75L) / ((long double)n + 0.5L));
        long double dp = 1.0L;
        for (int it = 0; it < 100; ++it) {
            long double p0 = 1.0L, p1 = t;  // P_0, P_1
            for (int k = 2; k <= n; ++k) {
                const long double pk = ((2.0L * k - 1.0L) * t * p1 - (k - 1.0L) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0L);  // P_n'(t)
            const long double dt = p1 / dp;
            t -= dt;
            if (fabsl(dt) <= 1e-19L * fabsl(t)) break;
        }
        x[i] = (double)t;
        w[i] = (double)(2.0L / ((1.0L - t * t) * dp * dp));
    }
}

__global__ void k_round_to_f32(const double2 *__restrict__ in, float2 *__restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

// FP64 spectra -> double-float pairs (GM_DF64): each part rounded to the nearest h + l
__global__ void k_split_df(const double2 *__restrict__ in, dfc *__restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        out[i] = c_make<dfc>(dfr(in[i].x), dfr(in[i].y));
    }
}

#define GM_TRY(x)                              \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) { err = e_; goto done; } \
    } while (0)

// Real even spectra of the station-centred generator (gravity with symmetric padding, Sec. 3,
// Eq. Tcircpadded): the generator e_r(dx, dy) = k_r(dx, dy) stored at (dx mod N'x, dy mod N'y) is
// the embedded generator t_r reflected and shifted by the padding, e[j] = t[(-j - pxl) mod N'], so
// E_r = w conj(T_r) with w = exp(+2 pi i (pxl kx / N'x + pyl ky / N'y)).  The gravity kernel is
// even in both offsets and the padding is the same on both sides, so E_r is real and even in ky:
// E[kx][r][ky] for ky <= N'y/2 is kept.  dev[0] / dev[1] receive the largest |Im| and the largest
// ky-mirror mismatch, and dev[2] the largest |E|, as the bit patterns of non-negative doubles.
template <typename Rout>
__global__ void k_real_even_spectrum(const double2 *__restrict__ S64, Rout *__restrict__ E, int Kx, int nz, int NPx,
                                     int NPy, int pxl, int pyl, unsigned long long *__restrict__ dev) {
    const int H = NPy / 2 + 1;
    const size_t total = (size_t)Kx * nz * H;
    double mi = 0, mm = 0, me = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int ky = (int)(i % H);
        const size_t kr = i / H;  // kx * nz + r
        const int kx = (int)(kr / nz);
        auto e_at = [&](int kyy) {
            double sx_, cx_, sy_, cy_;
            sincospi(2.0 * (double)(((long long)pxl * kx) % NPx) / NPx, &sx_, &cx_);
            sincospi(2.0 * (double)(((long long)pyl * kyy) % NPy) / NPy, &sy_, &cy_);
            const double wr = cx_ * cy_ - sx_ * sy_, wi = sx_ * cy_ + cx_ * sy_;
            const double2 t = S64[kr * NPy + kyy];
            // w * conj(t)
            return make_double2(wr * t.x + wi * t.y, wi * t.x - wr * t.y);
        };
        const double2 e = e_at(ky);
        const double2 f = e_at(ky == 0 ? 0 : NPy - ky);
        mi = fmax(mi, fmax(fabs(e.y), fabs(f.y)));
        mm = fmax(mm, fabs(e.x - f.x));
        me = fmax(me, fabs(e.x));
        E[i] = (Rout)e.x;
    }
    atomicMax(dev + 0, (unsigned long long)__double_as_longlong(mi));
    atomicMax(dev + 1, (unsigned long long)__double_as_longlong(mm));
    atomicMax(dev + 2, (unsigned long long)__double_as_longlong(me));
}

cudaError_t build_spectra(gm_plan *p, cudaStream_t s) {
    const Geo &g = p->geo;
    const int ncx = p->Nx + 1, ncy = p->Ny + 1;
    cudaError_t err = cudaSuccess;
    double *z = nullptr, *Q = nullptr, *T = nullptr;
    double2 *S64 = nullptr;
    void *tw64x = nullptr, *tw64y = nullptr;
    FftDesc fx64 = p->fx, fy64 = p->fy;
    const size_t nspec = (size_t)g.Kx * g.nz * g.NPy;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GM_TRY(cudaEventCreate(&e0));
    GM_TRY(cudaEventCreate(&e1));
    GM_TRY(cudaEventRecord(e0, s));
    GM_TRY(cudaMalloc(&z, sizeof(double) * (g.nz + 1)));
    GM_TRY(cudaMemcpyAsync(z, p->zplanes.data(), sizeof(double) * (g.nz + 1), cudaMemcpyHostToDevice, s));
    GM_TRY(cudaMalloc(&Q, sizeof(double) * (size_t)ncx * ncy * g.nz));
    GM_TRY(cudaMalloc(&T, sizeof(double) * (size_t)g.NPx * g.NPy * g.nz));
    GM_TRY(cudaMalloc(&S64, sizeof(double2) * nspec));
    if (p->precision == GM_F64) {
        tw64x = p->tw_x;
        tw64y = p->tw_y;
    } else {
        GM_TRY(make_twiddles(g.NPx, GM_F64, &tw64x));
        GM_TRY(make_twiddles(g.NPy, GM_F64, &tw64y));
    }
    fx64.tw = tw64x;
    fy64.tw = tw64y;
    {
        CornerArgs a;
        a.ncx = ncx; a.ncy = ncy; a.nz = g.nz;
        a.x0 = ((double)(-(g.sx - 1 + g.pxl)) - 0.5) * p->dx;
        a.y0 = ((double)(-(g.sy - 1 + g.pyl)) - 0.5) * p->dy;
        a.dx = p->dx; a.dy = p->dy; a.z = z; a.kind = p->kind;
        for (int k = 0; k < 5; ++k) a.c[k] = p->coef[k];
        dim3 blk(128), grd((ncx + 127) / 128, ncy, g.nz);
        k_corner_columns<<<grd, blk, 0, s>>>(Q, a);
        GM_TRY(cudaGetLastError());
    }
    {
        FarField f{};
        f.quad = p->kind == GM_GRAVITY ? 1 : 2;
        f.gap_cells = 2.5;
        {
            const double I = p->incl_deg * kPiSetup / 180.0, D = p->decl_deg * kPiSetup / 180.0;
            f.l = std::cos(I) * std::cos(D);
            f.m = std::cos(I) * std::sin(D);
            f.n = std::sin(I);
            f.H = p->F_nT / (4.0 * kPiSetup);
        }
        f.x0 = ((double)(-(g.sx - 1 + g.pxl)) - 0.5) * p->dx;
        f.y0 = ((double)(-(g.sy - 1 + g.pyl)) - 0.5) * p->dy;
        f.dx = p->dx;
        f.dy = p->dy;
        f.gamma = p->coef[0];
        f.z = z;
        gauss_legendre(8, f.g8.x, f.g8.w);
        gauss_legendre(6, f.g6.x, f.g6.w);
        gauss_legendre(5, f.g5.x, f.g5.w);
        gauss_legendre(4, f.g4.x, f.g4.w);
        dim3 blk(128), grd((g.NPx + 127) / 128, g.NPy, g.nz);
        k_generator<<<grd, blk, 0, s>>>(Q, T, g, ncx, ncy, f);
        GM_TRY(cudaGetLastError());
    }
    {
        // rows: T[r][vy][0:NPx] -> S64[kx][r][vy]
        dim3 grd((g.NPy + 1) / 2, g.nz);
        size_t sm = 2 * sizeof(double2) * g.NPx;
        GM_TRY(allow_smem(k_rows_r2c<double2, double>, sm));
        GM_TRY(allow_smem(k_cols_fft<double2>, 2 * sizeof(double2) * g.NPy));
        k_rows_r2c<double2, double><<<grd, 256, sm, s>>>(T, g.NPy, g.NPx, g.nz, S64, g.NPy, fx64, g.Kx);
        GM_TRY(cudaGetLastError());
        dim3 grd2(g.Kx, g.nz);
        size_t sm2 = 2 * sizeof(double2) * g.NPy;
        k_cols_fft<double2><<<grd2, 256, sm2, s>>>(S64, g.nz, g.NPy, fy64);
        GM_TRY(cudaGetLastError());
    }
    if (p->spec_real) {
        unsigned long long *dev = nullptr;
        unsigned long long hostv[3] = {0, 0, 0};
        GM_TRY(cudaMalloc(&dev, sizeof(hostv)));
        GM_TRY(cudaMemsetAsync(dev, 0, sizeof(hostv), s));
        if (p->precision == GM_F64)
            k_real_even_spectrum<double><<<1024, 256, 0, s>>>(S64, static_cast<double *>(p->spec), g.Kx, g.nz, g.NPx,
                                                              g.NPy, g.pxl, g.pyl, dev);
        else if (p->precision == GM_DF64)
            k_real_even_spectrum<dfr><<<1024, 256, 0, s>>>(S64, static_cast<dfr *>(p->spec), g.Kx, g.nz, g.NPx,
                                                           g.NPy, g.pxl, g.pyl, dev);
        else
            k_real_even_spectrum<float><<<1024, 256, 0, s>>>(S64, static_cast<float *>(p->spec), g.Kx, g.nz, g.NPx,
                                                             g.NPy, g.pxl, g.pyl, dev);
        err = cudaGetLastError();
        if (err == cudaSuccess) err = cudaMemcpyAsync(hostv, dev, sizeof(hostv), cudaMemcpyDeviceToHost, s);
        if (err == cudaSuccess) err = cudaStreamSynchronize(s);
        cudaFree(dev);
        GM_TRY(err);
        double v[3];
        std::memcpy(v, hostv, sizeof(v));
        // exact arithmetic makes Im and the mirror mismatch zero; FP64 rounding leaves ~1e-16 |E|
        if (!(v[0] <= 1e-9 * v[2]) || !(v[1] <= 1e-9 * v[2])) {
            err = cudaErrorInvalidValue;
            goto done;
        }
    } else if (p->precision == GM_F64) {
        GM_TRY(cudaMemcpyAsync(p->spec, S64, sizeof(double2) * nspec, cudaMemcpyDeviceToDevice, s));
    } else if (p->precision == GM_DF64) {
        k_split_df<<<1024, 256, 0, s>>>(S64, static_cast<dfc *>(p->spec), nspec);
        GM_TRY(cudaGetLastError());
    } else {
        k_round_to_f32<<<1024, 256, 0, s>>>(S64, reinterpret_cast<float2 *>(p->spec), nspec);
        GM_TRY(cudaGetLastError());
    }
    GM_TRY(cudaEventRecord(e1, s));
    GM_TRY(cudaStreamSynchronize(s));
    {
        float ms = 0;
        GM_TRY(cudaEventElapsedTime(&ms, e0, e1));
        p->setup_ms = ms;
    }
done:
    cudaStreamSynchronize(s);
    cudaFree(z);
    cudaFree(Q);
    cudaFree(T);
    cudaFree(S64);
    if (p->precision != GM_F64) {
        cudaFree(tw64x);
        cudaFree(tw64y);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return err;
}

}  // namespace gm
