// gm_fast_impl.cuh -- launch wrappers of the register-codelet kernels (gm_fast.cuh) for one FFT
// length, and the per-length function tables (XOps for the row direction, YOps for the column
// direction) that the fast_*.cu translation units instantiate over the length ladder.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "gm_fast.cuh"
#include "gm_fast_ops.h"
#include "gm_plan.h"

namespace gm {
namespace {

constexpr int kPairs = 8;   // two-row transforms per row-kernel CTA (many rows)
constexpr int kLstep = kColLayerStep;

// Row kernels with few CTAs' worth of rows use one-warp CTAs of a single two-row transform.
inline bool few_rows(int rows, int nlayers) {
    return (long long)((rows + 2 * kPairs - 1) / (2 * kPairs)) * nlayers < 2LL * sm_count();
}

template <int R1> constexpr int cols_per_cta() { return 256 / R1 > 0 ? 256 / R1 : 1; }

// ---- x-direction (rows): r2c with radices (X1, X2), c2r with (X2, X1)
template <typename R, int X1, int X2, int PAIRS, int THREADS>
cudaError_t rows_r2c_p(const io_t<R> *in, int rows, int row_len, int nlayers, cpx_t<R> *out, int out_rows,
                       const void *tw, cudaStream_t s) {
    using C = cpx_t<R>;
    const size_t sm = sizeof(C) * (PAIRS * fast::Ex<X1, X2>::value);
    auto k = fast::k_rows_r2c<C, io_t<R>, X1, X2, PAIRS, THREADS>;
    cudaError_t e = allow_smem(k, sm);
    if (e != cudaSuccess) return e;
    dim3 grd((rows + 2 * PAIRS - 1) / (2 * PAIRS), nlayers);
    e = launch_pdl(k, grd, dim3(THREADS), sm, s, in, rows, row_len, nlayers, out, out_rows, static_cast<const C *>(tw));
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <typename R, int X1, int X2>
cudaError_t rows_r2c(const io_t<R> *in, int rows, int row_len, int nlayers, cpx_t<R> *out, int out_rows,
                     const void *tw, cudaStream_t s) {
    static_assert(X1 <= 32 && X2 <= 32, "one-warp CTAs hold one item of each pass per thread");
    // (double-float builds only the many-rows form: its straight-line code is large to compile)
    if constexpr (!std::is_same<R, dfr>::value)
        if (few_rows(rows, nlayers)) return rows_r2c_p<R, X1, X2, 1, 32>(in, rows, row_len, nlayers, out, out_rows, tw, s);
    return rows_r2c_p<R, X1, X2, kPairs, 256>(in, rows, row_len, nlayers, out, out_rows, tw, s);
}

template <typename R, int X1, int X2, int PAIRS, int THREADS>
cudaError_t rows_c2r_p(const cpx_t<R> *in, long long ld_k, long long ld_layer, long long ld_row, int rows,
                       int nlayers, io_t<R> *out, int row_len_out, double scale, const void *tw, bool discard,
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
    const size_t sm = sizeof(C) * PAIRS * fast::C2rRegion<X2, X1>::value;
    auto k = fast::k_rows_c2r<C, io_t<R>, X2, X1, PAIRS, THREADS>;
    cudaError_t e = allow_smem(k, sm);
    if (e != cudaSuccess) return e;
    dim3 grd((rows + 2 * PAIRS - 1) / (2 * PAIRS), nlayers);
    e = launch_pdl(k, grd, dim3(THREADS), sm, s, in, ld_k, ld_layer, ld_row, rows, out, row_len_out, scale,
                   static_cast<const C *>(tw), disc);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <typename R, int X1, int X2>
cudaError_t rows_c2r(const cpx_t<R> *in, long long ld_k, long long ld_layer, long long ld_row, int rows,
                     int nlayers, io_t<R> *out, int row_len_out, double scale, const void *tw, bool discard,
                     cudaStream_t s) {
    if constexpr (!std::is_same<R, dfr>::value)
        if (few_rows(rows, nlayers))
            return rows_c2r_p<R, X1, X2, 1, 32>(in, ld_k, ld_layer, ld_row, rows, nlayers, out, row_len_out, scale,
                                                tw, discard, s);
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

// shared memory of the column kernels: the N-entry twiddle table, the per-pass tables (one for the
// forward kernel, two for the transpose kernel) and the exchanges
template <typename R, int Y1, int Y2>
constexpr size_t fwd_mac_smem_c() {
    constexpr int tables = fast::pass_tables<cpx_t<R>>() ? 2 : 1;
    return sizeof(cpx_t<R>) * (tables * Y1 * Y2 + cols_per_cta<Y1>() * kLstep * fast::Ex<Y1, Y2>::value);
}
template <typename R, int Y1, int Y2>
constexpr size_t tr_smem_c() {
    constexpr int a = fast::Ex<Y1, Y2>::value, b = fast::Ex<Y2, Y1>::value;
    constexpr int tables = fast::pass_tables<cpx_t<R>>() ? 3 : 1;
    return sizeof(cpx_t<R>) * (tables * Y1 * Y2 + cols_per_cta<Y1>() * kLstep * (a > b ? a : b));
}
template <typename R, int Y1, int Y2>
size_t fwd_mac_smem(int) { return fwd_mac_smem_c<R, Y1, Y2>(); }
template <typename R, int Y1, int Y2>
size_t tr_smem() { return tr_smem_c<R, Y1, Y2>(); }

// The spectrum form of a column kernel: fixed at compile time for FP32 (one kernel per form), chosen
// at run time for FP64 and double-float (one kernel for both forms, half the compile time).
template <typename R> constexpr int spec_mode(bool real) {
    return std::is_same<R, float>::value ? (real ? 1 : 0) : 2;
}
template <typename R, int Y1, int Y2, bool REAL>
const void *fwd_kernel() {
    using CC = ColCfg<R, Y1, Y2>;
    using C = cpx_t<R>;
    return (const void *)fast::k_cols_fwd_mac<C, Y1, Y2, CC::COLS, kLstep, CC::T_FWD, spec_mode<R>(REAL),
                                              fast::col_min_blocks<C>(fwd_mac_smem_c<R, Y1, Y2>())>;
}
template <typename R, int Y1, int Y2, bool REAL>
const void *tr_kernel() {
    using CC = ColCfg<R, Y1, Y2>;
    using C = cpx_t<R>;
    return (const void *)fast::k_cols_tr<C, Y1, Y2, CC::COLS_TR, kLstep, CC::T_TR, spec_mode<R>(REAL),
                                         fast::col_min_blocks<C>(tr_smem_c<R, Y1, Y2>())>;
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
                                       int, const C *, int, int, int, const C *)>(
        const_cast<void *>(p->spec_real ? fwd_kernel<R, Y1, Y2, true>() : fwd_kernel<R, Y1, Y2, false>()));
    cudaError_t e = allow_smem(k, sm);
    if (e != cudaSuccess) return e;
    dim3 grd((g.Kx + COLS - 1) / COLS, p->fast_groups_fwd);
    e = launch_pdl(k, grd, dim3(T), sm, s, A, S, part, B, static_cast<unsigned int *>(p->work_counters), g.Kx, g.nz,
                   g.ny, g.nyp, g.sy, p->fast_lpg_fwd, p->fast_groups_fwd, static_cast<const C *>(p->tw_y),
                   p->spec_real ? 1 : 0, g.pxl, g.pyl, static_cast<const C *>(p->tw_x));
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <typename R, int Y1, int Y2>
cudaError_t cols_tr(const gm_plan *p, const cpx_t<R> *D1, const cpx_t<R> *S, cpx_t<R> *A2, cudaStream_t s) {
    using C = cpx_t<R>;
    using CC = ColCfg<R, Y1, Y2>;
    constexpr int COLS = CC::COLS_TR, T = CC::T_TR;
    const Geo &g = p->geo;
    const size_t sm = tr_smem<R, Y1, Y2>();
    auto k = reinterpret_cast<void (*)(const C *, const C *, C *, int, int, int, int, int, int, const C *, int, int,
                                       int, const C *)>(
        const_cast<void *>(p->spec_real ? tr_kernel<R, Y1, Y2, true>() : tr_kernel<R, Y1, Y2, false>()));
    cudaError_t e = allow_smem(k, sm);
    if (e != cudaSuccess) return e;
    dim3 grd((g.Kx + COLS - 1) / COLS, p->fast_groups_tr);
    e = launch_pdl(k, grd, dim3(T), sm, s, D1, S, A2, g.Kx, g.nz, g.ny, g.nyp, g.sy, p->fast_lpg_tr,
                   static_cast<const C *>(p->tw_y), p->spec_real ? 1 : 0, g.pxl, g.pyl,
                   static_cast<const C *>(p->tw_x));
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <typename R, int X1, int X2>
XOps<R> make_xops() {
    XOps<R> o;
    o.r2c = rows_r2c<R, X1, X2>;
    o.c2r = rows_c2r<R, X1, X2>;
    return o;
}

template <typename R, int Y1, int Y2>
YOps<R> make_yops() {
    using CC = ColCfg<R, Y1, Y2>;
    YOps<R> o;
    o.fwd_mac = cols_fwd_mac<R, Y1, Y2>;
    o.tr = cols_tr<R, Y1, Y2>;
    o.cols = CC::COLS;
    o.cols_tr = CC::COLS_TR;
    o.block_fwd = CC::T_FWD;
    o.block_tr = CC::T_TR;
    o.smem_fwd = fwd_mac_smem<R, Y1, Y2>(0);
    o.smem_tr = tr_smem<R, Y1, Y2>();
    o.kern_fwd[0] = fwd_kernel<R, Y1, Y2, false>();
    o.kern_fwd[1] = fwd_kernel<R, Y1, Y2, true>();
    o.kern_tr[0] = tr_kernel<R, Y1, Y2, false>();
    o.kern_tr[1] = tr_kernel<R, Y1, Y2, true>();
    return o;
}

}  // namespace
}  // namespace gm
