// apply_fast.cu -- the register-codelet apply path (gm_fast.cuh) for the FFT lengths it is
// instantiated for; any other length uses the generic kernels of apply.cu.
//
// forward  d = G m:   rows r2c (K4) -> column FFT x depth-MAC over layer groups (K5)
//                     -> sum of groups + inverse column FFT (K5b) -> rows c2r + window (K6)
// transpose m' = G^T d: rows r2c of d (K7) -> column FFT of d, then per layer conj(S) x and
//                     inverse column FFT (K8) -> rows c2r + window (K9)
#include <cstdint>
#include <cuda_runtime.h>

#include <algorithm>

#include "gm_fast.cuh"
#include "gm_plan.h"

namespace gm {

namespace {

constexpr int kPairs = 8;   // two-row transforms per row-kernel CTA (many rows)
constexpr int kLstep = 2;   // layers per step in the column kernels

// Row kernels with few CTAs' worth of rows use one-warp CTAs of a single two-row transform.
inline bool few_rows(int rows, int nlayers) {
    return (long long)((rows + 2 * kPairs - 1) / (2 * kPairs)) * nlayers < 2LL * sm_count();
}

template <int R1> constexpr int cols_per_cta() { return 256 / R1 > 0 ? 256 / R1 : 1; }

// ---- x-direction (rows): r2c with radices (X1, X2), c2r with (X2, X1)
template <typename R, int X1, int X2, int PAIRS, int THREADS>
cudaError_t rows_r2c_p(const R *in, int rows, int row_len, int nlayers, cpx_t<R> *out, int out_rows,
                       const void *tw, cudaStream_t s) {
    using C = cpx_t<R>;
    const size_t sm = sizeof(C) * (PAIRS * fast::Ex<X1, X2>::value);
    auto k = fast::k_rows_r2c<C, R, X1, X2, PAIRS, THREADS>;
    cudaError_t e = allow_smem(k, sm);
    if (e != cudaSuccess) return e;
    dim3 grd((rows + 2 * PAIRS - 1) / (2 * PAIRS), nlayers);
    k<<<grd, THREADS, sm, s>>>(in, rows, row_len, nlayers, out, out_rows, static_cast<const C *>(tw));
    return cudaGetLastError();
}

template <typename R, int X1, int X2>
cudaError_t rows_r2c(const R *in, int rows, int row_len, int nlayers, cpx_t<R> *out, int out_rows,
                     const void *tw, cudaStream_t s) {
    static_assert(X1 <= 32 && X2 <= 32, "one-warp CTAs hold one item of each pass per thread");
    if (few_rows(rows, nlayers)) return rows_r2c_p<R, X1, X2, 1, 32>(in, rows, row_len, nlayers, out, out_rows, tw, s);
    return rows_r2c_p<R, X1, X2, kPairs, 256>(in, rows, row_len, nlayers, out, out_rows, tw, s);
}

template <typename R, int X1, int X2, int PAIRS, int THREADS>
cudaError_t rows_c2r_p(const cpx_t<R> *in, long long ld_k, long long ld_layer, long long ld_row, int rows,
                       int nlayers, R *out, int row_len_out, double scale, const void *tw, bool discard,
                       cudaStream_t s) {
    using C = cpx_t<R>;
    constexpr int N = X1 * X2, Kx = N / 2 + 1;
    // the block's run of 2*PAIRS rows per (k, layer) must be whole, aligned 128-byte lines
    constexpr long long LINE = 128 / (long long)sizeof(C);
    const int disc = (discard && ld_row == 1 && (2 * PAIRS) % LINE == 0 && ld_k % LINE == 0 &&
                      ld_layer % LINE == 0 && reinterpret_cast<uintptr_t>(in) % 128 == 0)
                         ? 1
                         : 0;
    // inverse radices (X2, X1): pass-2 items j < X2 write X2-wide coalesced rows
    const size_t sm = sizeof(C) * (2 * PAIRS * Kx + PAIRS * fast::Ex<X2, X1>::value);
    auto k = fast::k_rows_c2r<C, R, X2, X1, PAIRS, THREADS>;
    cudaError_t e = allow_smem(k, sm);
    if (e != cudaSuccess) return e;
    dim3 grd((rows + 2 * PAIRS - 1) / (2 * PAIRS), nlayers);
    k<<<grd, THREADS, sm, s>>>(in, ld_k, ld_layer, ld_row, rows, out, row_len_out, scale,
                               static_cast<const C *>(tw), disc);
    return cudaGetLastError();
}

template <typename R, int X1, int X2>
cudaError_t rows_c2r(const cpx_t<R> *in, long long ld_k, long long ld_layer, long long ld_row, int rows,
                     int nlayers, R *out, int row_len_out, double scale, const void *tw, bool discard,
                     cudaStream_t s) {
    if (few_rows(rows, nlayers))
        return rows_c2r_p<R, X1, X2, 1, 32>(in, ld_k, ld_layer, ld_row, rows, nlayers, out, row_len_out, scale, tw,
                                            discard, s);
    return rows_c2r_p<R, X1, X2, kPairs, 256>(in, ld_k, ld_layer, ld_row, rows, nlayers, out, row_len_out, scale,
                                              tw, discard, s);
}

// ---- y-direction (columns): forward radices (Y1, Y2)
template <int Y1> constexpr int cols_threads() { return (cols_per_cta<Y1>() * Y1 + 31) / 32 * 32; }

template <typename R, int Y1, int Y2> struct ColCfg {
    static constexpr int COLS = cols_per_cta<Y1>();
    static constexpr int T_FWD = cols_threads<Y1>();
    static constexpr int COLS_TR = cols_per_cta<Y1>();
    static constexpr int T_TR = cols_threads<Y1>();
};

template <typename R, int Y1, int Y2>
size_t fwd_mac_smem(int) {
    return sizeof(cpx_t<R>) * (Y1 * Y2 + cols_per_cta<Y1>() * kLstep * fast::Ex<Y1, Y2>::value);
}
template <typename R, int Y1, int Y2>
size_t tr_smem() {
    constexpr int a = fast::Ex<Y1, Y2>::value, b = fast::Ex<Y2, Y1>::value;
    return sizeof(cpx_t<R>) * (Y1 * Y2 + cols_per_cta<Y1>() * kLstep * (a > b ? a : b));
}

template <typename R, int Y1, int Y2>
const void *fwd_kernel() {
    using CC = ColCfg<R, Y1, Y2>;
    return (const void *)fast::k_cols_fwd_mac<cpx_t<R>, Y1, Y2, CC::COLS, kLstep, CC::T_FWD>;
}
template <typename R, int Y1, int Y2>
const void *tr_kernel() {
    using CC = ColCfg<R, Y1, Y2>;
    return (const void *)fast::k_cols_tr<cpx_t<R>, Y1, Y2, CC::COLS_TR, kLstep, CC::T_TR>;
}

template <typename R, int Y1, int Y2>
cudaError_t cols_fwd_mac(const gm_plan *p, const cpx_t<R> *A, const cpx_t<R> *S, cpx_t<R> *part, cpx_t<R> *B,
                         cudaStream_t s) {
    using C = cpx_t<R>;
    using CC = ColCfg<R, Y1, Y2>;
    constexpr int COLS = CC::COLS, T = CC::T_FWD;
    const Geo &g = p->geo;
    const size_t sm = fwd_mac_smem<R, Y1, Y2>(g.nyp);
    auto k = reinterpret_cast<void (*)(const C *, const C *, C *, C *, unsigned int *, int, int, int, int, int, int,
                                       int, const C *)>(const_cast<void *>(fwd_kernel<R, Y1, Y2>()));
    cudaError_t e = allow_smem(k, sm);
    if (e != cudaSuccess) return e;
    dim3 grd((g.Kx + COLS - 1) / COLS, p->fast_groups_fwd);
    k<<<grd, T, sm, s>>>(A, S, part, B, static_cast<unsigned int *>(p->work_counters), g.Kx, g.nz, g.ny, g.nyp,
                         g.sy, p->fast_lpg_fwd, p->fast_groups_fwd, static_cast<const C *>(p->tw_y));
    return cudaGetLastError();
}

template <typename R, int Y1, int Y2>
cudaError_t cols_tr(const gm_plan *p, const cpx_t<R> *D1, const cpx_t<R> *S, cpx_t<R> *A2, cudaStream_t s) {
    using C = cpx_t<R>;
    using CC = ColCfg<R, Y1, Y2>;
    constexpr int COLS = CC::COLS_TR, T = CC::T_TR;
    const Geo &g = p->geo;
    const size_t sm = tr_smem<R, Y1, Y2>();
    auto k = reinterpret_cast<void (*)(const C *, const C *, C *, int, int, int, int, int, int, const C *)>(
        const_cast<void *>(tr_kernel<R, Y1, Y2>()));
    cudaError_t e = allow_smem(k, sm);
    if (e != cudaSuccess) return e;
    dim3 grd((g.Kx + COLS - 1) / COLS, p->fast_groups_tr);
    k<<<grd, T, sm, s>>>(D1, S, A2, g.Kx, g.nz, g.ny, g.nyp, g.sy, p->fast_lpg_tr, static_cast<const C *>(p->tw_y));
    return cudaGetLastError();
}

// ---- dispatch by length
#define GM_X_SIZES(F) F(32, 4, 8) F(128, 8, 16) F(140, 7, 20) F(256, 16, 16) F(672, 21, 32)
#define GM_Y_SIZES(F) F(32, 4, 8) F(128, 8, 16) F(140, 14, 10) F(256, 16, 16) F(560, 35, 16)

bool x_supported(int N) {
#define F(n, a, b) if (N == n) return true;
    GM_X_SIZES(F)
#undef F
    return false;
}
bool y_supported(int N) {
#define F(n, a, b) if (N == n) return true;
    GM_Y_SIZES(F)
#undef F
    return false;
}

template <typename R>
cudaError_t x_r2c(int N, const R *in, int rows, int row_len, int nlayers, cpx_t<R> *out, int out_rows,
                  const void *tw, cudaStream_t s) {
#define F(n, a, b) if (N == n) return rows_r2c<R, a, b>(in, rows, row_len, nlayers, out, out_rows, tw, s);
    GM_X_SIZES(F)
#undef F
    return cudaErrorNotSupported;
}

template <typename R>
cudaError_t x_c2r(int N, const cpx_t<R> *in, long long ldk, long long ldl, long long ldr, int rows, int nlayers,
                  R *out, int row_len_out, double scale, const void *tw, bool discard, cudaStream_t s) {
#define F(n, a, b) \
    if (N == n) return rows_c2r<R, a, b>(in, ldk, ldl, ldr, rows, nlayers, out, row_len_out, scale, tw, discard, s);
    GM_X_SIZES(F)
#undef F
    return cudaErrorNotSupported;
}

template <typename R>
cudaError_t y_fwd_mac(const gm_plan *p, const cpx_t<R> *A, const cpx_t<R> *S, cpx_t<R> *part, cpx_t<R> *B,
                      cudaStream_t s) {
#define F(n, a, b) if (p->geo.NPy == n) return cols_fwd_mac<R, a, b>(p, A, S, part, B, s);
    GM_Y_SIZES(F)
#undef F
    return cudaErrorNotSupported;
}

template <typename R>
cudaError_t y_tr(const gm_plan *p, const cpx_t<R> *D1, const cpx_t<R> *S, cpx_t<R> *A2, cudaStream_t s) {
#define F(n, a, b) if (p->geo.NPy == n) return cols_tr<R, a, b>(p, D1, S, A2, s);
    GM_Y_SIZES(F)
#undef F
    return cudaErrorNotSupported;
}

template <typename R>
int y_cols_per_cta(int N, bool tr = false) {
#define F(n, a, b) if (N == n) return tr ? ColCfg<R, a, b>::COLS_TR : ColCfg<R, a, b>::COLS;
    GM_Y_SIZES(F)
#undef F
    return 1;
}

template <typename R>
int y_block(int N, bool tr) {
#define F(n, a, b) if (N == n) return tr ? ColCfg<R, a, b>::T_TR : ColCfg<R, a, b>::T_FWD;
    GM_Y_SIZES(F)
#undef F
    return 256;
}

template <typename R>
size_t y_smem(int N, bool tr, int nyp) {
#define F(n, a, b) if (N == n) return tr ? tr_smem<R, a, b>() : fwd_mac_smem<R, a, b>(nyp);
    GM_Y_SIZES(F)
#undef F
    return 0;
}

template <typename R>
const void *y_kernel(int N, bool tr) {
#define F(n, a, b)                                                                                     \
    if (N == n)                                                                                        \
        return tr ? tr_kernel<R, a, b>() : fwd_kernel<R, a, b>();
    GM_Y_SIZES(F)
#undef F
    return nullptr;
}

#define CK(x)                                  \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) return e_;      \
    } while (0)

template <typename R>
cudaError_t forward_fast_t(gm_plan *p, const R *m, R *d, cudaStream_t s, int *nl) {
    using C = cpx_t<R>;
    const Geo &g = p->geo;
    C *A = static_cast<C *>(p->work_big);
    C *B = static_cast<C *>(p->work_small);
    C *part = static_cast<C *>(p->work_part);
    const C *S = static_cast<const C *>(p->spec);
    int t = timing_begin(p, s, K_FWD_ROWS);
    CK(x_r2c<R>(g.NPx, m, g.ny, g.nx, g.nz, A, g.nyp, p->tw_x, s));
    timing_end(p, s, t);
    t = timing_begin(p, s, K_FWD_COLS);
    CK(y_fwd_mac<R>(p, A, S, part, B, s));
    timing_end(p, s, t);
    t = timing_begin(p, s, K_FWD_C2R);
    // B is [kx][j]: element (k, row j) at k*sy + j
    CK(x_c2r<R>(g.NPx, B, g.sy, 0, 1, g.sy, 1, d, g.sx, 1.0 / ((double)g.NPx * g.NPy), p->tw_x, false, s));
    timing_end(p, s, t);
    *nl = 3;
    return cudaSuccess;
}

template <typename R>
cudaError_t transpose_fast_t(gm_plan *p, const R *d, R *m, cudaStream_t s, int *nl) {
    using C = cpx_t<R>;
    const Geo &g = p->geo;
    C *D1 = static_cast<C *>(p->work_small);
    C *A2 = static_cast<C *>(p->work_big);
    const C *S = static_cast<const C *>(p->spec);
    int t = timing_begin(p, s, K_TR_ROWS);
    CK(x_r2c<R>(g.NPx, d, g.sy, g.sx, 1, D1, g.sy, p->tw_x, s));
    timing_end(p, s, t);
    t = timing_begin(p, s, K_TR_COLS);
    CK(y_tr<R>(p, D1, S, A2, s));
    timing_end(p, s, t);
    t = timing_begin(p, s, K_TR_C2R);
    // A2 is [kx][r][q] with column pitch nyp: element (k, layer r, row q) at (k*nz + r)*nyp + q
    // A2 is dead once read: its lines are dropped from L2 instead of being written back
    CK(x_c2r<R>(g.NPx, A2, (long long)g.nz * g.nyp, g.nyp, 1, g.ny, g.nz, m, g.nx, 1.0 / ((double)g.NPx * g.NPy),
                p->tw_x, true, s));
    timing_end(p, s, t);
    *nl = 3;
    return cudaSuccess;
}

// Layers per CTA group so that (column groups x layer groups) fills the GPU about once.
template <typename R>
void choose_groups(const gm_plan *p, bool tr, int *groups, int *lpg) {
    const Geo &g = p->geo;
    int dev = 0, sms = 1, occ = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int cols = y_cols_per_cta<R>(g.NPy, tr);
    const void *k = y_kernel<R>(g.NPy, tr);
    const size_t sm = y_smem<R>(g.NPy, tr, g.nyp);
    if (k) {
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, y_block<R>(g.NPy, tr), sm) != cudaSuccess ||
            occ < 1)
            occ = 1;
    }
    cudaGetLastError();
    const int colgroups = (g.Kx + cols - 1) / cols;
    int ng = std::max(1, std::min(g.nz, (sms * occ) / std::max(1, colgroups)));
    int per = (g.nz + ng - 1) / ng;
    *lpg = per;
    *groups = (g.nz + per - 1) / per;
}

}  // namespace

bool fast_path_supported(int NPx, int NPy) { return x_supported(NPx) && y_supported(NPy); }

int fast_column_groups(const gm_plan *p) {
    const int cols = p->precision == GM_F64 ? y_cols_per_cta<double>(p->geo.NPy) : y_cols_per_cta<float>(p->geo.NPy);
    return (p->geo.Kx + cols - 1) / cols;
}

void fast_plan_groups(gm_plan *p) {
    if (p->precision == GM_F64) {
        choose_groups<double>(p, false, &p->fast_groups_fwd, &p->fast_lpg_fwd);
        choose_groups<double>(p, true, &p->fast_groups_tr, &p->fast_lpg_tr);
    } else {
        choose_groups<float>(p, false, &p->fast_groups_fwd, &p->fast_lpg_fwd);
        choose_groups<float>(p, true, &p->fast_groups_tr, &p->fast_lpg_tr);
    }
}

cudaError_t launch_forward_fast(gm_plan *p, const void *m, void *d, cudaStream_t s, int *nl) {
    if (p->precision == GM_F64)
        return forward_fast_t<double>(p, static_cast<const double *>(m), static_cast<double *>(d), s, nl);
    return forward_fast_t<float>(p, static_cast<const float *>(m), static_cast<float *>(d), s, nl);
}

cudaError_t launch_transpose_fast(gm_plan *p, const void *d, void *m, cudaStream_t s, int *nl) {
    if (p->precision == GM_F64)
        return transpose_fast_t<double>(p, static_cast<const double *>(d), static_cast<double *>(m), s, nl);
    return transpose_fast_t<float>(p, static_cast<const float *>(d), static_cast<float *>(m), s, nl);
}

}  // namespace gm
