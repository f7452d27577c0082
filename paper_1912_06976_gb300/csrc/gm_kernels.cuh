// gm_kernels.cuh -- row and column FFT kernels of the 2-D transforms (Sec. 3, Eq. GrviaT).
//
// A 2-D FFT of a real N'_y x N'_x array is done as real-input FFTs along x
// (rows) followed by complex FFTs along y (columns) of the N'_x/2+1 kept
// x-frequencies.  Two real rows a, b share one complex FFT of a + i b; with
// Z = FFT(a + i b), FFT(a)[k] = (Z[k] + conj Z[-k]) / 2 and
// FFT(b)[k] = (Z[k] - conj Z[-k]) / (2i).  The inverse packs two Hermitian
// spectra X1 + i X2 into one inverse FFT whose real and imaginary parts are the
// two real rows.
#pragma once

#include "gm_common.cuh"

namespace gm {

// Real rows -> half spectra.  Block (pair, layer) transforms rows 2*pair and
// 2*pair+1 of `layer` of in[layer][row][0:row_len] (zero-padded to f.N) and
// writes out[k][layer][row] for k < Kx (out_rows = row stride of out).
template <typename C, typename Rin>
__global__ void k_rows_r2c(const Rin *__restrict__ in, int rows, int row_len, int nlayers,
                           C *__restrict__ out, int out_rows, FftDesc f, int Kx) {
    extern __shared__ unsigned char smem_raw[];
    C *b0 = reinterpret_cast<C *>(smem_raw);
    C *b1 = b0 + f.N;
    const int q0 = 2 * blockIdx.x;
    const int layer = blockIdx.y;
    const bool has1 = q0 + 1 < rows;
    const Rin *r0 = in + ((size_t)layer * rows + q0) * row_len;
    for (int n = threadIdx.x; n < f.N; n += blockDim.x) {
        C z;
        z.x = (n < row_len) ? (decltype(z.x))r0[n] : 0;
        z.y = (n < row_len && has1) ? (decltype(z.x))r0[row_len + n] : 0;
        b0[n] = z;
    }
    __syncthreads();
    C *Z = fft_block(b0, b1, 1, f.N, f, false);
    for (int k = threadIdx.x; k < Kx; k += blockDim.x) {
        C a = Z[k];
        C b = c_conj(Z[(f.N - k) % f.N]);
        C x1 = c_make<C>((a.x + b.x) * 0.5f, (a.y + b.y) * 0.5f);
        C x2 = c_make<C>((a.y - b.y) * 0.5f, -(a.x - b.x) * 0.5f);
        size_t o = ((size_t)k * nlayers + layer) * out_rows + q0;
        out[o] = x1;
        if (has1) out[o + 1] = x2;
    }
}

// Half spectra -> real rows.  Block (pair, layer) reads in[layer][row][0:Kx]
// for rows 2*pair, 2*pair+1, runs one inverse FFT and writes
// out[layer][row][0:row_len_out] = scale * (inverse transform)[0:row_len_out].
template <typename C, typename Rout>
__global__ void k_rows_c2r(const C *__restrict__ in, int rows, int nlayers, Rout *__restrict__ out,
                           int row_len_out, FftDesc f, int Kx, double scale) {
    extern __shared__ unsigned char smem_raw[];
    C *b0 = reinterpret_cast<C *>(smem_raw);
    C *b1 = b0 + f.N;
    const int q0 = 2 * blockIdx.x;
    const int layer = blockIdx.y;
    const bool has1 = q0 + 1 < rows;
    const C *r0 = in + ((size_t)layer * rows + q0) * Kx;
    const int half = f.N / 2;
    for (int n = threadIdx.x; n < f.N; n += blockDim.x) {
        const int kk = (n <= half) ? n : f.N - n;
        C x1 = r0[kk];
        C x2 = has1 ? r0[Kx + kk] : c_make<C>(0, 0);
        if (n > half) { x1 = c_conj(x1); x2 = c_conj(x2); }
        b0[n] = c_make<C>(x1.x - x2.y, x1.y + x2.x);
    }
    __syncthreads();
    C *z = fft_block(b0, b1, 1, f.N, f, true);
    Rout *o0 = out + ((size_t)layer * rows + q0) * row_len_out;
    for (int i = threadIdx.x; i < row_len_out; i += blockDim.x) {
        o0[i] = (Rout)(z[i].x * scale);
        if (has1) o0[row_len_out + i] = (Rout)(z[i].y * scale);
    }
}

// In-place complex FFT along the contiguous axis of data[col][layer][0:N]:
// block (col, layer) loads len_in values (zero-padded to N), transforms, stores N.
template <typename C>
__global__ void k_cols_fft(C *__restrict__ data, int nlayers, int len_in, FftDesc f) {
    extern __shared__ unsigned char smem_raw[];
    C *b0 = reinterpret_cast<C *>(smem_raw);
    C *b1 = b0 + f.N;
    C *col = data + ((size_t)blockIdx.x * nlayers + blockIdx.y) * f.N;
    for (int n = threadIdx.x; n < f.N; n += blockDim.x) b0[n] = (n < len_in) ? col[n] : c_make<C>(0, 0);
    __syncthreads();
    C *z = fft_block(b0, b1, 1, f.N, f, false);
    for (int n = threadIdx.x; n < f.N; n += blockDim.x) col[n] = z[n];
}

}  // namespace gm
