// apply_fast.cu -- the register-codelet apply path (gm_fast.cuh) for the FFT lengths of the
// ladder in gm_fast_ops.h; any other length uses the generic kernels of apply.cu.
//
// forward  d = G m:   rows r2c (K4) -> column FFT x depth-MAC over layer groups (K5)
//                     -> sum of groups + inverse column FFT (K5b) -> rows c2r + window (K6)
// transpose m' = G^T d: rows r2c of d (K7) -> column FFT of d, then per layer conj(S) x and
//                     inverse column FFT (K8) -> rows c2r + window (K9)
#include <cstdint>
#include <cstdlib>
#include <cuda_runtime.h>

#include <algorithm>

#include "gm_fast_ops.h"
#include "gm_plan.h"

namespace gm {

int fast_ladder_length(int n, bool y) {
    int best = 0;
#define F(len, a, b) \
    if (len >= n && (best == 0 || len < best)) best = len;
    if (y) {
        GM_Y_LADDER_A(F)
        GM_Y_LADDER_B(F)
    } else {
        GM_X_LADDER(F)
    }
#undef F
    return best;
}

namespace {

#define CK(x)                                  \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) return e_;      \
    } while (0)

template <typename R>
cudaError_t forward_fast_t(gm_plan *p, const io_t<R> *m, io_t<R> *d, cudaStream_t s, int *nl) {
    using C = cpx_t<R>;
    const Geo &g = p->geo;
    C *A = static_cast<C *>(p->work_big);
    C *B = static_cast<C *>(p->work_small);
    C *part = static_cast<C *>(p->work_part);
    const C *S = static_cast<const C *>(p->spec);
    const XOps<R> *xo = x_ops<R>(g.NPx);
    const YOps<R> *yo = y_ops<R>(g.NPy);
    if (!xo || !yo) return cudaErrorNotSupported;
    // (each launch is bracketed by timing_begin / timing_end, also when it fails)
    int t = timing_begin(p, s, K_FWD_ROWS);
    cudaError_t e = xo->r2c(m, g.ny, g.nx, g.nz, A, g.nyp, p->tw_x, s);
    timing_end(p, s, t);
    CK(e);
    t = timing_begin(p, s, K_FWD_COLS);
    e = yo->fwd_mac(p, A, S, part, B, s);
    timing_end(p, s, t);
    CK(e);
    t = timing_begin(p, s, K_FWD_C2R);
    // B is [kx][j]: element (k, row j) at k*sy + j
    e = xo->c2r(B, g.sy, 0, 1, g.sy, 1, d, g.sx, 1.0 / ((double)g.NPx * g.NPy), p->tw_x, false, s);
    timing_end(p, s, t);
    CK(e);
    *nl = 3;
    return cudaSuccess;
}

template <typename R>
cudaError_t transpose_fast_t(gm_plan *p, const io_t<R> *d, io_t<R> *m, cudaStream_t s, int *nl) {
    using C = cpx_t<R>;
    const Geo &g = p->geo;
    C *D1 = static_cast<C *>(p->work_small_tr);
    C *A2 = static_cast<C *>(p->work_big_tr);
    const C *S = static_cast<const C *>(p->spec);
    const XOps<R> *xo = x_ops<R>(g.NPx);
    const YOps<R> *yo = y_ops<R>(g.NPy);
    if (!xo || !yo) return cudaErrorNotSupported;
    int t = timing_begin(p, s, K_TR_ROWS);
    cudaError_t e = xo->r2c(d, g.sy, g.sx, 1, D1, g.sy, p->tw_x, s);
    timing_end(p, s, t);
    CK(e);
    t = timing_begin(p, s, K_TR_COLS);
    e = yo->tr(p, D1, S, A2, s);
    timing_end(p, s, t);
    CK(e);
    t = timing_begin(p, s, K_TR_C2R);
    // A2 is [kx][r][q] with column pitch nyp: element (k, layer r, row q) at (k*nz + r)*nyp + q
    // A2 is dead once read: its lines are dropped from L2 instead of being written back
    e = xo->c2r(A2, (long long)g.nz * g.nyp, g.nyp, 1, g.ny, g.nz, m, g.nx, 1.0 / ((double)g.NPx * g.NPy), p->tw_x,
                true, s);
    timing_end(p, s, t);
    CK(e);
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
    const YOps<R> *yo = y_ops<R>(g.NPy);
    const int cols = yo ? (tr ? yo->cols_tr : yo->cols) : 1;
    const int real = p->spec_real ? 1 : 0;
    const void *k = yo ? (tr ? yo->kern_tr[real] : yo->kern_fwd[real]) : nullptr;
    const size_t sm = yo ? (tr ? yo->smem_tr : yo->smem_fwd) : 0;
    if (k) {
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, tr ? yo->block_tr : yo->block_fwd, sm) !=
                cudaSuccess ||
            occ < 1)
            occ = 1;
    }
    cudaGetLastError();
    const int colgroups = (g.Kx + cols - 1) / cols;
    int ng = std::max(1, std::min(g.nz, (sms * occ) / std::max(1, colgroups)));
    int per = (g.nz + ng - 1) / ng;
    // The forward kernel transforms kColLayerStep layers per step: a one-layer group would leave
    // half of each step idle and double the partial sums its finishing blocks add up (measured on
    // 128 x 128 x 32 magnetic data: 20.4 us at one layer per group, 14.3 us at two).  The
    // transpose writes each layer on its own and is fastest at the fill-the-GPU choice.
    if (!tr) per = std::max(per, std::min(kColLayerStep, g.nz));
    // tuning override: layers per CTA group of the forward / transpose column kernels
    if (const char *ov = std::getenv(tr ? "GM_TR_LAYERS_PER_GROUP" : "GM_FWD_LAYERS_PER_GROUP"))
        if (std::atoi(ov) > 0) per = std::min(g.nz, std::atoi(ov));
    *lpg = per;
    *groups = (g.nz + per - 1) / per;
}

}  // namespace

bool fast_path_supported(int NPx, int NPy) { return x_ops_f32(NPx) != nullptr && y_ops<float>(NPy) != nullptr; }

int fast_column_groups(const gm_plan *p) {
    const int cols = p->precision == GM_F64    ? y_ops<double>(p->geo.NPy)->cols
                     : p->precision == GM_DF64 ? y_ops<dfr>(p->geo.NPy)->cols
                                               : y_ops<float>(p->geo.NPy)->cols;
    return (p->geo.Kx + cols - 1) / cols;
}

void fast_plan_groups(gm_plan *p) {
    if (p->precision == GM_F64) {
        choose_groups<double>(p, false, &p->fast_groups_fwd, &p->fast_lpg_fwd);
        choose_groups<double>(p, true, &p->fast_groups_tr, &p->fast_lpg_tr);
    } else if (p->precision == GM_DF64) {
        choose_groups<dfr>(p, false, &p->fast_groups_fwd, &p->fast_lpg_fwd);
        choose_groups<dfr>(p, true, &p->fast_groups_tr, &p->fast_lpg_tr);
    } else {
        choose_groups<float>(p, false, &p->fast_groups_fwd, &p->fast_lpg_fwd);
        choose_groups<float>(p, true, &p->fast_groups_tr, &p->fast_lpg_tr);
    }
}

cudaError_t launch_forward_fast(gm_plan *p, const void *m, void *d, cudaStream_t s, int *nl) {
    if (p->precision == GM_F64)
        return forward_fast_t<double>(p, static_cast<const double *>(m), static_cast<double *>(d), s, nl);
    if (p->precision == GM_DF64)
        return forward_fast_t<dfr>(p, static_cast<const double *>(m), static_cast<double *>(d), s, nl);
    return forward_fast_t<float>(p, static_cast<const float *>(m), static_cast<float *>(d), s, nl);
}

cudaError_t launch_transpose_fast(gm_plan *p, const void *d, void *m, cudaStream_t s, int *nl) {
    if (p->precision == GM_F64)
        return transpose_fast_t<double>(p, static_cast<const double *>(d), static_cast<double *>(m), s, nl);
    if (p->precision == GM_DF64)
        return transpose_fast_t<dfr>(p, static_cast<const double *>(d), static_cast<double *>(m), s, nl);
    return transpose_fast_t<float>(p, static_cast<const float *>(d), static_cast<float *>(m), s, nl);
}

}  // namespace gm
