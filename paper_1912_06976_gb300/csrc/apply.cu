// apply.cu -- forward and transpose products through the block-circulant embedding.
//
// Algorithm multbttb (App. B) with Eq. GrviaT, re-organised for one GPU:
//
// forward  d = G m (t = 1):
//   K4 row FFTs:  A[kx][r][q] = FFT_x(m[r][q][0:nx] zero-padded to N'_x)[kx]   (Eq. Wpadded)
//   K5 per x-frequency kx:  acc = SUM_r S[kx][r][:] * FFT_y(A[kx][r][0:ny] zero-padded to N'_y);
//      B[j][kx] = IFFT_y(acc)[j], j < sy.  The depth sum is taken in the frequency
//      domain (Sec. 5: G u = SUM_r G^(r) u_r and the FFT is linear), so one inverse
//      transform serves all layers.
//   K6 row inverse FFTs:  d[j][i] = IFFT_x(B[j][:])[i] / (N'_x N'_y), i < sx
//      (the top-left s_x x s_y block of Eq. GrviaT).
// transpose m' = G^T d (t = 2):
//   K7 row FFTs of d (Eq. WTpadded)  ->  D1[kx][j]
//   K8 per kx: Dh = FFT_y(D1[kx][0:sy]); for each r: A2[r][q][kx] = IFFT_y(conj(S[kx][r][:]) * Dh)[q], q < ny
//      (conj(S) is the spectrum of the transposed generator of Eqs. Ttran0 / Ttran,
//      because the generator is real)
//   K9 row inverse FFTs:  m'[r][q][p] = IFFT_x(A2[r][q][:])[p] / (N'_x N'_y), p < nx.
#include <cuda_runtime.h>

#include "gm_kernels.cuh"
#include "gm_plan.h"

namespace gm {

constexpr int kThreads = 256;

// K5: column FFTs + depth multiply-accumulate + one inverse column FFT.
template <typename C>
__global__ void k_fwd_cols_mac(const C *__restrict__ A, const C *__restrict__ S, C *__restrict__ B, Geo g,
                               FftDesc fy) {
    extern __shared__ unsigned char smem_raw[];
    const int N = fy.N;
    C *acc = reinterpret_cast<C *>(smem_raw);
    C *b0 = acc + N;
    C *b1 = b0 + N;
    const int kx = blockIdx.x;
    for (int n = threadIdx.x; n < N; n += blockDim.x) acc[n] = c_make<C>(0, 0);
    for (int r = 0; r < g.nz; ++r) {
        const C *col = A + ((size_t)kx * g.nz + r) * g.ny;
        for (int n = threadIdx.x; n < N; n += blockDim.x) b0[n] = (n < g.ny) ? col[n] : c_make<C>(0, 0);
        __syncthreads();
        C *X = fft_block(b0, b1, 1, N, fy, false);
        const C *Sr = S + ((size_t)kx * g.nz + r) * N;
        for (int n = threadIdx.x; n < N; n += blockDim.x) acc[n] = c_add(acc[n], c_mul(X[n], Sr[n]));
        __syncthreads();
    }
    C *y = fft_block(acc, b0, 1, N, fy, true);
    for (int j = threadIdx.x; j < g.sy; j += blockDim.x) B[(size_t)j * g.Kx + kx] = y[j];
}

// K8: one forward column FFT of the data, then per layer multiply by conj(S) and invert.
template <typename C>
__global__ void k_tr_cols(const C *__restrict__ D1, const C *__restrict__ S, C *__restrict__ A2, Geo g,
                          FftDesc fy) {
    extern __shared__ unsigned char smem_raw[];
    const int N = fy.N;
    C *dh = reinterpret_cast<C *>(smem_raw);
    C *b0 = dh + N;
    C *b1 = b0 + N;
    const int kx = blockIdx.x;
    const C *col = D1 + (size_t)kx * g.sy;
    for (int n = threadIdx.x; n < N; n += blockDim.x) b0[n] = (n < g.sy) ? col[n] : c_make<C>(0, 0);
    __syncthreads();
    C *X = fft_block(b0, b1, 1, N, fy, false);
    for (int n = threadIdx.x; n < N; n += blockDim.x) dh[n] = X[n];
    __syncthreads();
    for (int r = 0; r < g.nz; ++r) {
        const C *Sr = S + ((size_t)kx * g.nz + r) * N;
        for (int n = threadIdx.x; n < N; n += blockDim.x) b0[n] = c_mulc(dh[n], Sr[n]);
        __syncthreads();
        C *y = fft_block(b0, b1, 1, N, fy, true);
        for (int q = threadIdx.x; q < g.ny; q += blockDim.x) A2[((size_t)r * g.ny + q) * g.Kx + kx] = y[q];
        __syncthreads();
    }
}

template <typename R>
static cudaError_t forward_t(gm_plan *p, const R *m, R *d, cudaStream_t s, int *nl) {
    using C = cpx_t<R>;
    const Geo &g = p->geo;
    C *A = reinterpret_cast<C *>(p->work_big);
    C *B = reinterpret_cast<C *>(p->work_small);
    const C *S = reinterpret_cast<const C *>(p->spec);
    allow_smem(k_rows_r2c<C, R>, 2 * sizeof(C) * g.NPx);
    allow_smem(k_fwd_cols_mac<C>, 3 * sizeof(C) * g.NPy);
    allow_smem(k_rows_c2r<C, R>, 2 * sizeof(C) * g.NPx);
    int t = timing_begin(p, s, K_FWD_ROWS);
    k_rows_r2c<C, R><<<dim3((g.ny + 1) / 2, g.nz), kThreads, 2 * sizeof(C) * g.NPx, s>>>(
        m, g.ny, g.nx, g.nz, A, g.ny, p->fx, g.Kx);
    timing_end(p, s, t);
    t = timing_begin(p, s, K_FWD_COLS);
    k_fwd_cols_mac<C><<<g.Kx, kThreads, 3 * sizeof(C) * g.NPy, s>>>(A, S, B, g, p->fy);
    timing_end(p, s, t);
    t = timing_begin(p, s, K_FWD_C2R);
    k_rows_c2r<C, R><<<dim3((g.sy + 1) / 2, 1), kThreads, 2 * sizeof(C) * g.NPx, s>>>(
        B, g.sy, 1, d, g.sx, p->fx, g.Kx, 1.0 / ((double)g.NPx * g.NPy));
    timing_end(p, s, t);
    *nl = 3;
    return cudaGetLastError();
}

template <typename R>
static cudaError_t transpose_t(gm_plan *p, const R *d, R *m, cudaStream_t s, int *nl) {
    using C = cpx_t<R>;
    const Geo &g = p->geo;
    C *D1 = reinterpret_cast<C *>(p->work_small_tr);
    C *A2 = reinterpret_cast<C *>(p->work_big_tr);
    const C *S = reinterpret_cast<const C *>(p->spec);
    allow_smem(k_rows_r2c<C, R>, 2 * sizeof(C) * g.NPx);
    allow_smem(k_tr_cols<C>, 3 * sizeof(C) * g.NPy);
    allow_smem(k_rows_c2r<C, R>, 2 * sizeof(C) * g.NPx);
    int t = timing_begin(p, s, K_TR_ROWS);
    k_rows_r2c<C, R><<<dim3((g.sy + 1) / 2, 1), kThreads, 2 * sizeof(C) * g.NPx, s>>>(
        d, g.sy, g.sx, 1, D1, g.sy, p->fx, g.Kx);
    timing_end(p, s, t);
    t = timing_begin(p, s, K_TR_COLS);
    k_tr_cols<C><<<g.Kx, kThreads, 3 * sizeof(C) * g.NPy, s>>>(D1, S, A2, g, p->fy);
    timing_end(p, s, t);
    t = timing_begin(p, s, K_TR_C2R);
    k_rows_c2r<C, R><<<dim3((g.ny + 1) / 2, g.nz), kThreads, 2 * sizeof(C) * g.NPx, s>>>(
        A2, g.ny, g.nz, m, g.nx, p->fx, g.Kx, 1.0 / ((double)g.NPx * g.NPy));
    timing_end(p, s, t);
    *nl = 3;
    return cudaGetLastError();
}

cudaError_t launch_forward(gm_plan *p, const void *m, void *d, cudaStream_t s, int *nl) {
    if (p->fast) return launch_forward_fast(p, m, d, s, nl);
    if (p->precision == GM_F64)
        return forward_t<double>(p, static_cast<const double *>(m), static_cast<double *>(d), s, nl);
    return forward_t<float>(p, static_cast<const float *>(m), static_cast<float *>(d), s, nl);
}

cudaError_t launch_transpose(gm_plan *p, const void *d, void *m, cudaStream_t s, int *nl) {
    if (p->fast) return launch_transpose_fast(p, d, m, s, nl);
    if (p->precision == GM_F64)
        return transpose_t<double>(p, static_cast<const double *>(d), static_cast<double *>(m), s, nl);
    return transpose_t<float>(p, static_cast<const float *>(d), static_cast<float *>(m), s, nl);
}

}  // namespace gm
