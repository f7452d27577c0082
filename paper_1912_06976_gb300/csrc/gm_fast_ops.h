// gm_fast_ops.h -- function tables of the register-codelet apply path, one per FFT length of
// the ladder below and per precision.  A plan takes the smallest ladder length >= N'_min in each
// direction (when within 25% of the smallest even 7-smooth length); other lengths use the generic
// kernels.  Each row-direction entry (N, X1, X2) runs the r2c transform with radices (X1, X2) and
// the c2r transform with (X2, X1), both <= 32 (one lane per item); each column-direction entry
// (N, Y1, Y2) runs pass 1 with radix Y1 and keeps the Y2 pass-2 outputs in registers.
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

#include "gm_common.cuh"

struct gm_plan;

#define GM_X_LADDER(F)                                                                                           \
    F(32, 4, 8) F(48, 6, 8) F(64, 8, 8) F(80, 10, 8) F(96, 12, 8) F(112, 7, 16) F(128, 8, 16) F(140, 7, 20)        \
    F(160, 10, 16) F(192, 12, 16) F(224, 14, 16) F(256, 16, 16) F(288, 9, 32) F(320, 10, 32) F(384, 12, 32)        \
    F(448, 14, 32) F(512, 16, 32) F(560, 20, 28) F(576, 18, 32) F(640, 20, 32) F(672, 21, 32) F(768, 24, 32)       \
    F(896, 28, 32) F(1024, 32, 32)
#define GM_Y_LADDER_A(F)                                                                                         \
    F(32, 4, 8) F(48, 6, 8) F(64, 8, 8) F(80, 10, 8) F(96, 12, 8) F(112, 7, 16) F(128, 8, 16) F(140, 14, 10)       \
    F(160, 10, 16) F(192, 12, 16) F(224, 14, 16) F(256, 16, 16)
#define GM_Y_LADDER_B(F)                                                                                         \
    F(288, 18, 16) F(320, 20, 16) F(384, 24, 16) F(448, 28, 16) F(512, 32, 16) F(560, 35, 16) F(576, 24, 24)     \
    F(640, 32, 20) F(672, 28, 24) F(768, 32, 24)

namespace gm {

constexpr int kColLayerStep = 2;  // layers per step in the column kernels

template <typename R> struct XOps {
    cudaError_t (*r2c)(const io_t<R> *in, int rows, int row_len, int nlayers, cpx_t<R> *out, int out_rows, const void *tw,
                       cudaStream_t s);
    cudaError_t (*c2r)(const cpx_t<R> *in, long long ld_k, long long ld_layer, long long ld_row, int rows,
                       int nlayers, io_t<R> *out, int row_len_out, double scale, const void *tw, bool discard,
                       cudaStream_t s);
};

template <typename R> struct YOps {
    cudaError_t (*fwd_mac)(const gm_plan *p, const cpx_t<R> *A, const cpx_t<R> *S, cpx_t<R> *part, cpx_t<R> *B,
                           cudaStream_t s);
    cudaError_t (*tr)(const gm_plan *p, const cpx_t<R> *D1, const cpx_t<R> *S, cpx_t<R> *A2, cudaStream_t s);
    int cols, cols_tr, block_fwd, block_tr;
    size_t smem_fwd, smem_tr;
    const void *kern_fwd[2], *kern_tr[2];  // [0] complex spectra, [1] real even spectra
};

// nullptr when the length is not on the ladder (defined in fast_x_*.cu, fast_y_*.cu)
const XOps<float> *x_ops_f32(int N);
const XOps<double> *x_ops_f64(int N);
const YOps<float> *y_ops_f32(int N);
const YOps<double> *y_ops_f64(int N);
const YOps<float> *y_ops_f32_large(int N);
const YOps<double> *y_ops_f64_large(int N);
const XOps<dfr> *x_ops_df(int N);
const YOps<dfr> *y_ops_df(int N);

template <typename R> const XOps<R> *x_ops(int N);
template <> inline const XOps<float> *x_ops<float>(int N) { return x_ops_f32(N); }
template <> inline const XOps<double> *x_ops<double>(int N) { return x_ops_f64(N); }
template <> inline const XOps<dfr> *x_ops<dfr>(int N) { return x_ops_df(N); }
template <typename R> const YOps<R> *y_ops(int N);
template <> inline const YOps<float> *y_ops<float>(int N) {
    const YOps<float> *o = y_ops_f32(N);
    return o ? o : y_ops_f32_large(N);
}
template <> inline const YOps<double> *y_ops<double>(int N) {
    const YOps<double> *o = y_ops_f64(N);
    return o ? o : y_ops_f64_large(N);
}

template <> inline const YOps<dfr> *y_ops<dfr>(int N) { return y_ops_df(N); }

// smallest ladder length >= n in the row (y = false) or column (y = true) direction, or 0
int fast_ladder_length(int n, bool y);

}  // namespace gm
