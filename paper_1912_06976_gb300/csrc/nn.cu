// nn.cu -- the learned warm start: a 2-D convolutional encoder and a 3-D convolutional
// decoder that map a data grid d[sy][sx] to a model m[nz][ny][nx], trained on (model, data)
// pairs made by the fast forward operator; its prediction starts the Tikhonov CGLS.
//
// Layers (NCDHW, x fastest; 2-D layers are 3-D layers of depth 1):
//   encoder  E0 conv(1,3,3)   1 -> 32   S x S        ReLU
//            E1..E4 conv(1,3,3) stride (1,2,2): 32 -> 64 -> 128 -> 256 -> 512, down to S/16 ReLU
//   reshape  512 x 1 x (S/16)^2  ->  128 x 4 x (S/16)^2   (channel c = 4 c' + z; no data movement)
//   decoder  D1 up (2,2,2), conv(3,3,3) 128 -> 64  ReLU     D2 up (2,2,2), conv 64 -> 32 ReLU
//            D3 up (1,2,2), conv 32 -> 16 ReLU             D4 up (1,2,2), conv 16 -> 1 (linear)
//   output   1 x 16 x S x S
// Weights: FP32 master copies updated by Adam; the convolution kernels read a BF16 copy and
// accumulate in FP32.  Every kernel here is plain CUDA-core code: direct convolutions with
// weights broadcast across a block and several output channels per thread.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/gm_warmstart.h"

namespace gm {
namespace nn {

struct ConvDims {
    int N, CI, CO;
    int ID, IH, IW;  // input (already up-sampled)
    int OD, OH, OW;
    int KD, KH, KW;
    int SD, SH, SW;
    int PD, PH, PW;
};

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

constexpr int kChunk = 8;     // input (forward) or output (data gradient) channels staged per round
constexpr int kMaxTaps = 27;  // 3 x 3 x 3

// Stage w[co0 + t][ci][tap] (forward, TRANS = false) or w[co][ci0 + t][tap] (data gradient,
// TRANS = true) for the kChunk channels c0.. of the summed axis into smem[c][tap][t] as float.
template <int CT, bool TRANS>
__device__ __forceinline__ void stage_weights(float *sm, const __nv_bfloat16 *__restrict__ w, const ConvDims &d,
                                              int fixed0, int c0, int K) {
    const int n = kChunk * K * CT;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int t = e % CT, tap = (e / CT) % K, c = e / (CT * K);
        const int sc = c0 + c, fc = fixed0 + t;  // summed channel, fixed channel
        float v = 0.f;
        if (!TRANS) {
            if (sc < d.CI && fc < d.CO) v = bf(w[((size_t)fc * d.CI + sc) * K + tap]);
        } else {
            if (sc < d.CO && fc < d.CI) v = bf(w[((size_t)sc * d.CI + fc) * K + tap]);
        }
        sm[e] = v;
    }
}

// out[n][co][o] = b[co] + SUM_ci SUM_taps w[co][ci][tap] in[n][ci][o*s + tap - p]; optional ReLU.
// Block: blockDim.x output positions of one example, CT output channels per thread.
template <int CT>
__global__ void k_conv_fwd(const float *__restrict__ in, const __nv_bfloat16 *__restrict__ w,
                           const float *__restrict__ b, float *__restrict__ out, ConvDims d, int relu) {
    __shared__ __align__(16) float sw[kChunk * kMaxTaps * CT];
    const int osz = d.OD * d.OH * d.OW;
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    const int co0 = blockIdx.y * CT;
    const int n = blockIdx.z;
    const bool active = o < osz;
    const int oo = active ? o : 0;
    const int ox = oo % d.OW, oy = (oo / d.OW) % d.OH, oz = oo / (d.OW * d.OH);
    const int K = d.KD * d.KH * d.KW;
    float acc[CT];
#pragma unroll
    for (int t = 0; t < CT; ++t) acc[t] = (co0 + t < d.CO) ? b[co0 + t] : 0.f;
    const size_t isz = (size_t)d.ID * d.IH * d.IW;
    const float *inn = in + (size_t)n * d.CI * isz;
    for (int c0 = 0; c0 < d.CI; c0 += kChunk) {
        __syncthreads();
        stage_weights<CT, false>(sw, w, d, co0, c0, K);
        __syncthreads();
        if (!active) continue;
        const int cn = min(kChunk, d.CI - c0);
        for (int c = 0; c < cn; ++c) {
            const float *inc = inn + (size_t)(c0 + c) * isz;
            const float *swc = sw + c * K * CT;
            for (int kz = 0; kz < d.KD; ++kz) {
                const int iz = oz * d.SD + kz - d.PD;
                if (iz < 0 || iz >= d.ID) continue;
                for (int ky = 0; ky < d.KH; ++ky) {
                    const int iy = oy * d.SH + ky - d.PH;
                    if (iy < 0 || iy >= d.IH) continue;
                    const float *row = inc + ((size_t)iz * d.IH + iy) * d.IW;
                    const float *wt = swc + ((kz * d.KH + ky) * d.KW) * CT;
                    for (int kx = 0; kx < d.KW; ++kx) {
                        const int ix = ox * d.SW + kx - d.PW;
                        if (ix < 0 || ix >= d.IW) continue;
                        const float x = row[ix];
#pragma unroll
                        for (int t = 0; t < CT; ++t) acc[t] = fmaf(wt[kx * CT + t], x, acc[t]);
                    }
                }
            }
        }
    }
    if (!active) return;
#pragma unroll
    for (int t = 0; t < CT; ++t)
        if (co0 + t < d.CO) {
            float v = acc[t];
            if (relu) v = fmaxf(v, 0.f);
            out[((size_t)n * d.CO + co0 + t) * osz + o] = v;
        }
}

// din[n][ci][i] = SUM_co SUM_taps w[co][ci][tap] g[n][co][(i + p - tap) / s]  (exact division only)
template <int CT>
__global__ void k_conv_bwd_data(const float *__restrict__ g, const __nv_bfloat16 *__restrict__ w,
                                float *__restrict__ din, ConvDims d) {
    __shared__ __align__(16) float sw[kChunk * kMaxTaps * CT];
    const int isz = d.ID * d.IH * d.IW;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int ci0 = blockIdx.y * CT;
    const int n = blockIdx.z;
    const bool active = i < isz;
    const int ii = active ? i : 0;
    const int ix = ii % d.IW, iy = (ii / d.IW) % d.IH, iz = ii / (d.IW * d.IH);
    const int K = d.KD * d.KH * d.KW;
    const size_t osz = (size_t)d.OD * d.OH * d.OW;
    float acc[CT];
#pragma unroll
    for (int t = 0; t < CT; ++t) acc[t] = 0.f;
    const float *gn = g + (size_t)n * d.CO * osz;
    for (int c0 = 0; c0 < d.CO; c0 += kChunk) {
        __syncthreads();
        stage_weights<CT, true>(sw, w, d, ci0, c0, K);
        __syncthreads();
        if (!active) continue;
        const int cn = min(kChunk, d.CO - c0);
        for (int c = 0; c < cn; ++c) {
            const float *gc = gn + (size_t)(c0 + c) * osz;
            const float *swc = sw + c * K * CT;
            for (int kz = 0; kz < d.KD; ++kz) {
                const int tz = iz + d.PD - kz;
                if (tz < 0 || tz % d.SD) continue;
                const int oz = tz / d.SD;
                if (oz >= d.OD) continue;
                for (int ky = 0; ky < d.KH; ++ky) {
                    const int ty = iy + d.PH - ky;
                    if (ty < 0 || ty % d.SH) continue;
                    const int oy = ty / d.SH;
                    if (oy >= d.OH) continue;
                    const float *row = gc + ((size_t)oz * d.OH + oy) * d.OW;
                    const float *wt = swc + ((kz * d.KH + ky) * d.KW) * CT;
                    for (int kx = 0; kx < d.KW; ++kx) {
                        const int tx = ix + d.PW - kx;
                        if (tx < 0 || tx % d.SW) continue;
                        const int ox = tx / d.SW;
                        if (ox >= d.OW) continue;
                        const float gv = row[ox];
#pragma unroll
                        for (int t = 0; t < CT; ++t) acc[t] = fmaf(wt[kx * CT + t], gv, acc[t]);
                    }
                }
            }
        }
    }
    if (!active) return;
#pragma unroll
    for (int t = 0; t < CT; ++t)
        if (ci0 + t < d.CI) din[((size_t)n * d.CI + ci0 + t) * isz + i] = acc[t];
}


// Partial weight and bias gradients over one chunk of the (example, output position) pairs:
//   dwp[chunk][co][ci][kz][ky][kx] = SUM g[n][co][o] in[n][ci][o*s + (kz,ky,kx) - p]
//   dbp[chunk][co]                 = SUM g[n][co][o]                 (blocks with ci = kz = 0)
// Block (co tile of COT channels, ci, kz) x chunk; each thread keeps COT x 9 (ky, kx) sums in
// registers over its positions (per position: COT gradient loads, 9 input loads, 9 COT FMAs),
// then the block reduces them with warp shuffles and shared memory.
template <int COT>
__global__ void __launch_bounds__(256) k_conv_wgrad(const float *__restrict__ g, const float *__restrict__ in,
                                                    float *__restrict__ dwp, float *__restrict__ dbp, ConvDims d,
                                                    int chunk) {
    int bx = blockIdx.x;
    const int kz = bx % d.KD;
    bx /= d.KD;
    const int ci = bx % d.CI;
    const int co0 = (bx / d.CI) * COT;
    const int osz = d.OD * d.OH * d.OW;
    const long long total = (long long)d.N * osz;
    const long long beg = (long long)blockIdx.y * chunk;
    const long long end = min(total, beg + chunk);
    const size_t isz = (size_t)d.ID * d.IH * d.IW;
    float acc[COT][9], accb[COT];
#pragma unroll
    for (int t = 0; t < COT; ++t) {
        accb[t] = 0.f;
#pragma unroll
        for (int q = 0; q < 9; ++q) acc[t][q] = 0.f;
    }
    for (long long e = beg + threadIdx.x; e < end; e += blockDim.x) {
        const int n = (int)(e / osz), o = (int)(e - (long long)n * osz);
        const int ox = o % d.OW, oy = (o / d.OW) % d.OH, oz = o / (d.OW * d.OH);
        float gv[COT];
#pragma unroll
        for (int t = 0; t < COT; ++t) {
            gv[t] = (co0 + t < d.CO) ? g[((size_t)n * d.CO + co0 + t) * osz + o] : 0.f;
            accb[t] += gv[t];
        }
        const int iz = oz * d.SD + kz - d.PD;
        if (iz < 0 || iz >= d.ID) continue;
        const float *plane = in + ((size_t)n * d.CI + ci) * isz + (size_t)iz * d.IH * d.IW;
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
            const int iy = oy * d.SH + ky - d.PH;
            const bool vy = iy >= 0 && iy < d.IH;
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                const int ix = ox * d.SW + kx - d.PW;
                const float x = (vy && ix >= 0 && ix < d.IW) ? plane[(size_t)iy * d.IW + ix] : 0.f;
#pragma unroll
                for (int t = 0; t < COT; ++t) acc[t][ky * 3 + kx] = fmaf(gv[t], x, acc[t][ky * 3 + kx]);
            }
        }
    }
    // block reduction of the COT * 10 sums
    constexpr int NV = COT * 10;
    __shared__ float red[8][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
#pragma unroll
    for (int t = 0; t < COT; ++t) {
#pragma unroll
        for (int q = 0; q < 10; ++q) {
            float v = q < 9 ? acc[t][q] : accb[t];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) red[warp][t * 10 + q] = v;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NV; i += blockDim.x) {
        float v = 0.f;
        for (int w = 0; w < nwarp; ++w) v += red[w][i];
        const int t = i / 10, q = i % 10, co = co0 + t;
        if (co >= d.CO) continue;
        if (q < 9) {
            dwp[(size_t)blockIdx.y * d.CO * d.CI * d.KD * 9 + (((size_t)co * d.CI + ci) * d.KD + kz) * 9 + q] = v;
        } else if (ci == 0 && kz == 0) {
            dbp[(size_t)blockIdx.y * d.CO + co] = v;
        }
    }
}

// dst[i] = SUM_c part[c][i] (fixed order), c < chunks
__global__ void k_sum_chunks(const float *__restrict__ part, float *__restrict__ dst, size_t n, int chunks) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int c = 0; c < chunks; ++c) s += part[(size_t)c * n + i];
        dst[i] = s;
    }
}

// nearest up-sampling by (fz, fy, fx): out[n][c][z][y][x] = in[n][c][z/fz][y/fy][x/fx]
__global__ void k_upsample(const float *__restrict__ in, float *__restrict__ out, int NC, int D, int H, int W, int fz,
                           int fy, int fx) {
    const size_t OD = (size_t)D * fz, OH = (size_t)H * fy, OW = (size_t)W * fx;
    const size_t tot = (size_t)NC * OD * OH * OW;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x) {
        const size_t x = i % OW, y = (i / OW) % OH, z = (i / (OW * OH)) % OD, c = i / (OW * OH * OD);
        out[i] = in[((c * D + z / fz) * H + y / fy) * W + x / fx];
    }
}

// adjoint of k_upsample: in[n][c][z][y][x] = SUM of out over its (fz, fy, fx) block
__global__ void k_upsample_bwd(const float *__restrict__ gout, float *__restrict__ gin, int NC, int D, int H, int W,
                               int fz, int fy, int fx) {
    const size_t tot = (size_t)NC * D * H * W;
    const size_t OH = (size_t)H * fy, OW = (size_t)W * fx, OD = (size_t)D * fz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x) {
        const size_t x = i % W, y = (i / W) % H, z = (i / ((size_t)W * H)) % D, c = i / ((size_t)W * H * D);
        float s = 0.f;
        for (int a = 0; a < fz; ++a)
            for (int bq = 0; bq < fy; ++bq)
                for (int e = 0; e < fx; ++e)
                    s += gout[((c * OD + z * fz + a) * OH + y * fy + bq) * OW + x * fx + e];
        gin[i] = s;
    }
}

// g *= (out > 0)
__global__ void k_relu_mask(float *__restrict__ g, const float *__restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (!(out[i] > 0.f)) g[i] = 0.f;
}

// mean squared error: g = 2 (p - t) / n; part[block] = partial SUM (p - t)^2
__global__ void k_mse(const float *__restrict__ p, const float *__restrict__ t, float *__restrict__ g,
                      float *__restrict__ part, size_t n) {
    float s = 0.f;
    const float inv = 2.f / (float)n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float r = p[i] - t[i];
        s += r * r;
        g[i] = inv * r;
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    __shared__ float red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.f;
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}

__global__ void k_loss_final(const float *__restrict__ part, int nb, float *__restrict__ loss, float inv_n) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        float s = 0.f;
        for (int i = 0; i < nb; ++i) s += part[i];
        *loss = s * inv_n;
    }
}

// Adam with bias correction; w (FP32 master) and its BF16 copy
__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m1,
                       float *__restrict__ m2, __nv_bfloat16 *__restrict__ wb, size_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.f - b1) * gi;
        const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = v;
        const float wi = w[i] - lr * (a / c1) / (sqrtf(v / c2) + eps);
        w[i] = wi;
        if (wb) wb[i] = __float2bfloat16(wi);
    }
}

// r = a * r - x (the scaled data misfit in_scale (G m - d), x = in_scale d); part[block] = SUM r^2
__global__ void k_misfit(float *__restrict__ r, const float *__restrict__ x, float a, float *__restrict__ part,
                         size_t n) {
    float s = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float v = a * r[i] - x[i];
        r[i] = v;
        s += v * v;
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    __shared__ float red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.f;
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}

// y += a * x
__global__ void k_axpy(float *__restrict__ y, const float *__restrict__ x, float a, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = fmaf(a, x[i], y[i]);
}

__global__ void k_to_bf16(const float *__restrict__ w, __nv_bfloat16 *__restrict__ wb, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        wb[i] = __float2bfloat16(w[i]);
}

__global__ void k_scale(const float *__restrict__ x, float *__restrict__ y, size_t n, float a) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = a * x[i];
}

// y[b][e] = a * x[idx[b]][e] (idx == nullptr: x[b][e]), e < per: the minibatch gather of training.
// An index outside [0, count) gives a zero example and sets *bad.
__global__ void k_scale_gather(const float *__restrict__ x, const int *__restrict__ idx, int count,
                               float *__restrict__ y, size_t per, int batch, float a, int *__restrict__ bad) {
    const size_t n = per * (size_t)batch;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t b = i / per, e = i - b * per;
        const long long src = idx ? (long long)idx[b] : (long long)b;
        if (src < 0 || src >= count) {
            y[i] = 0.f;
            if (e == 0) atomicExch(bad, 1);
        } else {
            y[i] = a * x[(size_t)src * per + e];
        }
    }
}

// ------------------------------------------------------------------------------------------
struct Layer {
    ConvDims d;          // N is set per call
    int up[3];           // nearest up-sampling factors of the layer input (z, y, x)
    int in_d, in_h, in_w;  // input before up-sampling
    bool relu;
    size_t w_off, b_off, nw;
    bool upsampled() const { return up[0] * up[1] * up[2] > 1; }
    size_t in_low(int N) const { return (size_t)N * d.CI * in_d * in_h * in_w; }
    size_t in_up(int N) const { return (size_t)N * d.CI * d.ID * d.IH * d.IW; }
    size_t out(int N) const { return (size_t)N * d.CO * d.OD * d.OH * d.OW; }
};

}  // namespace nn
}  // namespace gm

// Buffers, for layer l (L layers): x[l] its input before up-sampling (x[0] the scaled data,
// x[l] = output of layer l - 1), u[l] its up-sampled input, y the network output; gx, gu, gy the
// loss gradients with respect to the same tensors.
struct gm_net {
    int device = 0;
    int S = 64, D = 16, max_batch = 0;
    std::vector<gm::nn::Layer> layers;
    size_t nparam = 0;
    float *w = nullptr, *gw = nullptr, *m1 = nullptr, *m2 = nullptr;
    __nv_bfloat16 *wb = nullptr;
    std::vector<float *> x, u, gx, gu;
    float *y = nullptr, *gy = nullptr, *target = nullptr;
    float *wpart = nullptr;  // per-chunk weight-gradient partials
    float *loss_part = nullptr, *loss = nullptr;
    gm_handle op = nullptr;    // FP32 operator of the data term (not owned)
    float lambda = 0.f;
    float *misfit = nullptr, *gt = nullptr, *mpred = nullptr;  // data-term buffers, allocated on first use
    float *loss_data = nullptr, *loss_data_part = nullptr;
    float *loss_pair = nullptr;  // pinned: last (model term, data term)
    int *bad_index = nullptr;  // set by the gather kernel when an index is out of range
    int *bad_host = nullptr;   // pinned
    float in_scale = 1.f, out_scale = 1.f;
    long long step = 0;
    int last_launches = 0;
};

namespace {

using gm::nn::ConvDims;
using gm::nn::Layer;

constexpr int kWgChunk = 8192;  // (example, output position) pairs per weight-gradient block
constexpr int kWgCo = 8;        // output channels per weight-gradient block
constexpr int kLossBlocks = 1024;
constexpr int kCT = 8;          // output channels per thread in the convolution kernels

thread_local char g_nn_msg[256] = "";

gm_status nn_fail(gm_status st, const char *msg) {
    std::strncpy(g_nn_msg, msg, sizeof(g_nn_msg) - 1);
    g_nn_msg[sizeof(g_nn_msg) - 1] = 0;
    return st;
}

unsigned long long splitmix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void build_layers(gm_net *net) {
    const int S = net->S, s = S / 16;
    auto add = [&](int ci, int co, int in_d, int in_h, int in_w, int uz, int uy, int ux, int kd, int sh, bool relu) {
        Layer l{};
        l.up[0] = uz;
        l.up[1] = uy;
        l.up[2] = ux;
        l.in_d = in_d;
        l.in_h = in_h;
        l.in_w = in_w;
        ConvDims &d = l.d;
        d.CI = ci;
        d.CO = co;
        d.ID = in_d * uz;
        d.IH = in_h * uy;
        d.IW = in_w * ux;
        d.KD = kd;
        d.KH = 3;
        d.KW = 3;
        d.SD = 1;
        d.SH = sh;
        d.SW = sh;
        d.PD = kd / 2;
        d.PH = 1;
        d.PW = 1;
        d.OD = (d.ID + 2 * d.PD - d.KD) / d.SD + 1;
        d.OH = (d.IH + 2 * d.PH - d.KH) / d.SH + 1;
        d.OW = (d.IW + 2 * d.PW - d.KW) / d.SW + 1;
        l.relu = relu;
        l.nw = (size_t)co * ci * kd * 9;
        net->layers.push_back(l);
    };
    add(1, 32, 1, S, S, 1, 1, 1, 1, 1, true);                 // E0
    add(32, 64, 1, S, S, 1, 1, 1, 1, 2, true);                // E1
    add(64, 128, 1, S / 2, S / 2, 1, 1, 1, 1, 2, true);       // E2
    add(128, 256, 1, S / 4, S / 4, 1, 1, 1, 1, 2, true);      // E3
    add(256, 512, 1, S / 8, S / 8, 1, 1, 1, 1, 2, true);      // E4
    add(128, 64, 4, s, s, 2, 2, 2, 3, 1, true);               // D1 (input: E4 output read as 128 x 4)
    add(64, 32, 8, 2 * s, 2 * s, 2, 2, 2, 3, 1, true);        // D2
    add(32, 16, 16, 4 * s, 4 * s, 1, 2, 2, 3, 1, true);       // D3
    add(16, 1, 16, 8 * s, 8 * s, 1, 2, 2, 3, 1, false);       // D4
    size_t off = 0;
    for (auto &l : net->layers) {
        l.w_off = off;
        off += l.nw;
        l.b_off = off;
        off += l.d.CO;
    }
    net->nparam = off;
}

int grid1(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 4096); }

cudaError_t launch_conv_fwd(const float *in, const __nv_bfloat16 *w, const float *b, float *out, const ConvDims &d,
                            bool relu, cudaStream_t s) {
    const int osz = d.OD * d.OH * d.OW;
    const int bx = osz >= 128 ? 128 : 32;
    const dim3 grd((osz + bx - 1) / bx, (d.CO + kCT - 1) / kCT, d.N);
    gm::nn::k_conv_fwd<kCT><<<grd, bx, 0, s>>>(in, w, b, out, d, relu ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_conv_bwd_data(const float *g, const __nv_bfloat16 *w, float *din, const ConvDims &d,
                                 cudaStream_t s) {
    const int isz = d.ID * d.IH * d.IW;
    const int bx = isz >= 128 ? 128 : 32;
    const dim3 grd((isz + bx - 1) / bx, (d.CI + kCT - 1) / kCT, d.N);
    gm::nn::k_conv_bwd_data<kCT><<<grd, bx, 0, s>>>(g, w, din, d);
    return cudaGetLastError();
}

// f(in_scale d) into net->y; returns the launches made
int forward_all(gm_net *net, const float *d_dev, const int *idx, int count, int N, cudaStream_t s) {
    int nl = 0;
    const size_t per = (size_t)net->S * net->S;
    gm::nn::k_scale_gather<<<grid1(per * N), 256, 0, s>>>(d_dev, idx, count, net->x[0], per, N, net->in_scale,
                                                          net->bad_index);
    ++nl;
    const size_t L = net->layers.size();
    for (size_t k = 0; k < L; ++k) {
        Layer l = net->layers[k];
        l.d.N = N;
        const float *src = net->x[k];
        if (l.upsampled()) {
            gm::nn::k_upsample<<<grid1(l.in_up(N)), 256, 0, s>>>(src, net->u[k], N * l.d.CI, l.in_d, l.in_h, l.in_w,
                                                                 l.up[0], l.up[1], l.up[2]);
            ++nl;
            src = net->u[k];
        }
        float *dst = (k + 1 < L) ? net->x[k + 1] : net->y;
        launch_conv_fwd(src, net->wb + l.w_off, net->w + l.b_off, dst, l.d, l.relu, s);
        ++nl;
    }
    return nl;
}

// parameter gradient into net->gw from the output gradient in net->gy; returns the launches made
int backward_all(gm_net *net, int N, cudaStream_t s) {
    int nl = 0;
    const size_t L = net->layers.size();
    float *g = net->gy;
    for (size_t k = L; k-- > 0;) {
        Layer l = net->layers[k];
        l.d.N = N;
        const float *out = (k + 1 < L) ? net->x[k + 1] : net->y;
        if (l.relu) {
            gm::nn::k_relu_mask<<<grid1(l.out(N)), 256, 0, s>>>(g, out, l.out(N));
            ++nl;
        }
        const float *in = l.upsampled() ? net->u[k] : net->x[k];
        const long long total = (long long)N * l.d.OD * l.d.OH * l.d.OW;
        const int chunks = (int)((total + kWgChunk - 1) / kWgChunk);
        float *dwp = net->wpart;
        float *dbp = net->wpart + (size_t)chunks * l.nw;
        gm::nn::k_conv_wgrad<kWgCo><<<dim3(((l.d.CO + kWgCo - 1) / kWgCo) * l.d.CI * l.d.KD, chunks), 256, 0, s>>>(
            g, in, dwp, dbp, l.d, kWgChunk);
        gm::nn::k_sum_chunks<<<grid1(l.nw), 256, 0, s>>>(dwp, net->gw + l.w_off, l.nw, chunks);
        gm::nn::k_sum_chunks<<<grid1(l.d.CO), 256, 0, s>>>(dbp, net->gw + l.b_off, l.d.CO, chunks);
        nl += 3;
        if (k == 0) break;  // no gradient with respect to the data
        if (l.upsampled()) {
            launch_conv_bwd_data(g, net->wb + l.w_off, net->gu[k], l.d, s);
            gm::nn::k_upsample_bwd<<<grid1(l.in_low(N)), 256, 0, s>>>(net->gu[k], net->gx[k], N * l.d.CI, l.in_d,
                                                                      l.in_h, l.in_w, l.up[0], l.up[1], l.up[2]);
            nl += 2;
        } else {
            launch_conv_bwd_data(g, net->wb + l.w_off, net->gx[k], l.d, s);
            ++nl;
        }
        g = net->gx[k];
    }
    return nl;
}

void free_net(gm_net *n) {
    if (!n) return;
    for (float *p : {n->w, n->gw, n->m1, n->m2, n->y, n->gy, n->target, n->wpart, n->loss_part, n->loss, n->misfit,
                     n->gt, n->mpred, n->loss_data, n->loss_data_part})
        cudaFree(p);
    if (n->loss_pair) cudaFreeHost(n->loss_pair);
    cudaFree(n->wb);
    cudaFree(n->bad_index);
    if (n->bad_host) cudaFreeHost(n->bad_host);
    for (auto *v : {&n->x, &n->u, &n->gx, &n->gu})
        for (float *p : *v) cudaFree(p);
    delete n;
}

bool dev_alloc(float **p, size_t elems, size_t *total) {
    *total += elems * sizeof(float);
    return cudaMalloc(p, elems * sizeof(float)) == cudaSuccess;
}

}  // namespace

extern "C" {

gm_net_handle gm_net_create(int grid, int depth, int max_batch, unsigned long long seed) {
    if (grid < 16 || grid > 1024 || grid % 16 || depth != 16 || max_batch < 1 || max_batch > 65535) {
        nn_fail(GM_EINVAL, "gm_net_create: grid must be a multiple of 16 in [16, 1024], depth 16, "
                           "1 <= max_batch <= 65535");
        return nullptr;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        nn_fail(GM_ENODEV, "gm_net_create: no CUDA device");
        return nullptr;
    }
    gm_net *net = new (std::nothrow) gm_net();
    if (!net) {
        nn_fail(GM_ENOMEM, "gm_net_create: host allocation failed");
        return nullptr;
    }
    net->device = dev;
    net->S = grid;
    net->D = depth;
    net->max_batch = max_batch;
    build_layers(net);
    const size_t P = net->nparam, L = net->layers.size();
    const int B = max_batch;
    size_t total = 0;
    bool ok = dev_alloc(&net->w, P, &total) && dev_alloc(&net->gw, P, &total) && dev_alloc(&net->m1, P, &total) &&
              dev_alloc(&net->m2, P, &total) && cudaMalloc(&net->wb, 2 * P) == cudaSuccess;
    net->x.assign(L, nullptr);
    net->u.assign(L, nullptr);
    net->gx.assign(L, nullptr);
    net->gu.assign(L, nullptr);
    size_t wpart = 0;
    for (size_t k = 0; ok && k < L; ++k) {
        const Layer &l = net->layers[k];
        ok = dev_alloc(&net->x[k], l.in_low(B), &total) && dev_alloc(&net->gx[k], l.in_low(B), &total);
        if (ok && l.upsampled()) ok = dev_alloc(&net->u[k], l.in_up(B), &total) && dev_alloc(&net->gu[k], l.in_up(B), &total);
        const long long pairs = (long long)B * l.d.OD * l.d.OH * l.d.OW;
        const size_t chunks = (size_t)((pairs + kWgChunk - 1) / kWgChunk);
        wpart = std::max(wpart, chunks * (l.nw + l.d.CO));
    }
    const size_t nout = net->layers.back().out(B);
    ok = ok && dev_alloc(&net->y, nout, &total) && dev_alloc(&net->gy, nout, &total) &&
         dev_alloc(&net->target, nout, &total) && dev_alloc(&net->wpart, wpart, &total) &&
         dev_alloc(&net->loss_part, kLossBlocks, &total) && dev_alloc(&net->loss, 1, &total) &&
         cudaMalloc(&net->bad_index, sizeof(int)) == cudaSuccess &&
         cudaMallocHost(&net->bad_host, sizeof(int)) == cudaSuccess &&
         cudaMallocHost(&net->loss_pair, 2 * sizeof(float)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_net(net);
        nn_fail(GM_ENOMEM, "gm_net_create: device allocation failed");
        return nullptr;
    }
    // He-uniform weights (bound sqrt(6 / fan_in); sqrt(3 / fan_in) for the linear output layer)
    std::vector<float> host(P, 0.f);
    for (size_t k = 0; k < L; ++k) {
        const Layer &l = net->layers[k];
        const double fan_in = (double)l.d.CI * l.d.KD * l.d.KH * l.d.KW;
        const double bound = std::sqrt((l.relu ? 6.0 : 3.0) / fan_in);
        for (size_t i = 0; i < l.nw; ++i) {
            const unsigned long long r = splitmix64(seed * 0x100000001B3ull + l.w_off + i);
            const double u01 = (double)(r >> 11) * (1.0 / 9007199254740992.0);
            host[l.w_off + i] = (float)((2.0 * u01 - 1.0) * bound);
        }
    }
    cudaError_t e = cudaMemcpy(net->w, host.data(), 4 * P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(net->m1, 0, 4 * P);
    if (e == cudaSuccess) e = cudaMemset(net->m2, 0, 4 * P);
    if (e == cudaSuccess) e = cudaMemset(net->gw, 0, 4 * P);
    if (e == cudaSuccess) e = cudaMemset(net->bad_index, 0, sizeof(int));
    net->loss_pair[0] = net->loss_pair[1] = 0.f;
    if (e == cudaSuccess) {
        gm::nn::k_to_bf16<<<grid1(P), 256>>>(net->w, net->wb, P);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_net(net);
        nn_fail(GM_ECUDA, "gm_net_create: initialisation failed");
        return nullptr;
    }
    return net;
}

gm_status gm_net_destroy(gm_net_handle net) {
    if (!net) return GM_OK;
    cudaDeviceSynchronize();
    free_net(net);
    return GM_OK;
}

int64_t gm_net_num_params(gm_net_handle net) { return net ? (int64_t)net->nparam : -1; }

gm_status gm_net_set_scales(gm_net_handle net, float in_scale, float out_scale) {
    if (!net || !(in_scale > 0.f) || !(out_scale > 0.f) || !std::isfinite(in_scale) || !std::isfinite(out_scale))
        return nn_fail(GM_EINVAL, "gm_net_set_scales: scales must be finite and > 0");
    net->in_scale = in_scale;
    net->out_scale = out_scale;
    return GM_OK;
}

gm_status gm_net_forward(gm_net_handle net, const float *d_dev, float *m_dev, int batch, void *stream) {
    if (!net || !d_dev || !m_dev || batch < 1 || batch > net->max_batch)
        return nn_fail(GM_EINVAL, "gm_net_forward: null pointer or batch outside [1, max_batch]");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int nl = forward_all(net, d_dev, nullptr, batch, batch, s);
    const size_t nout = net->layers.back().out(batch);
    gm::nn::k_scale<<<grid1(nout), 256, 0, s>>>(net->y, m_dev, nout, net->out_scale);
    net->last_launches = nl + 1;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GM_OK : nn_fail(GM_ECUDA, cudaGetErrorString(e));
}

gm_status gm_net_train_step(gm_net_handle net, const float *d_dev, const float *m_dev, int count,
                            const int32_t *index_dev, int batch, float lr, float *loss_host, void *stream) {
    if (!net || !d_dev || !m_dev || batch < 1 || batch > net->max_batch || !(lr >= 0.f) || !std::isfinite(lr) ||
        count < 1 || (!index_dev && batch > count))
        return nn_fail(GM_EINVAL, "gm_net_train_step: null pointer, batch outside [1, max_batch], batch > count "
                                  "without an index, or bad lr");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int nl = forward_all(net, d_dev, index_dev, count, batch, s);
    const size_t nout = net->layers.back().out(batch);
    gm::nn::k_scale_gather<<<grid1(nout), 256, 0, s>>>(m_dev, index_dev, count, net->target, nout / batch, batch,
                                                       1.f / net->out_scale, net->bad_index);
    gm::nn::k_mse<<<kLossBlocks, 256, 0, s>>>(net->y, net->target, net->gy, net->loss_part, nout);
    gm::nn::k_loss_final<<<1, 32, 0, s>>>(net->loss_part, kLossBlocks, net->loss, 1.f / (float)nout);
    nl += 3;
    if (net->lambda > 0.f) {
        // lambda mean((in_scale (G m - d))^2), m = out_scale y; its gradient 2 lambda / (batch nd)
        // in_scale out_scale G^T r with respect to y, through this library's own FP32 products
        const size_t per_m = nout / batch, per_d = (size_t)net->S * net->S, nd = per_d * batch;
        gm::nn::k_scale<<<grid1(nout), 256, 0, s>>>(net->y, net->mpred, nout, net->out_scale);
        for (int b = 0; b < batch; ++b) {
            const gm_status st = apply_forward(net->op, net->mpred + b * per_m, net->misfit + b * per_d, s);
            if (st != GM_OK) return nn_fail(st, "gm_net_train_step: forward product of the data term failed");
            nl += gm_last_launch_count(net->op);
        }
        gm::nn::k_misfit<<<kLossBlocks, 256, 0, s>>>(net->misfit, net->x[0], net->in_scale, net->loss_data_part, nd);
        gm::nn::k_loss_final<<<1, 32, 0, s>>>(net->loss_data_part, kLossBlocks, net->loss_data, 1.f / (float)nd);
        for (int b = 0; b < batch; ++b) {
            const gm_status st = apply_transpose(net->op, net->misfit + b * per_d, net->gt + b * per_m, s);
            if (st != GM_OK) return nn_fail(st, "gm_net_train_step: transpose product of the data term failed");
            nl += gm_last_launch_count(net->op);
        }
        const float coef = 2.f * net->lambda / (float)nd * net->in_scale * net->out_scale;
        gm::nn::k_axpy<<<grid1(nout), 256, 0, s>>>(net->gy, net->gt, coef, nout);
        nl += 4;
    }
    nl += backward_all(net, batch, s);
    if (lr > 0.f) {
        net->step += 1;
        const double b1 = 0.9, b2 = 0.999;
        const float c1 = (float)(1.0 - std::pow(b1, (double)net->step));
        const float c2 = (float)(1.0 - std::pow(b2, (double)net->step));
        gm::nn::k_adam<<<grid1(net->nparam), 256, 0, s>>>(net->w, net->gw, net->m1, net->m2, net->wb, net->nparam, lr,
                                                          (float)b1, (float)b2, 1e-8f, c1, c2);
        ++nl;
    }
    net->last_launches = nl;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && loss_host) {
        int bad = 0;
        net->loss_pair[1] = 0.f;
        e = cudaMemcpyAsync(net->loss_pair, net->loss, sizeof(float), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && net->lambda > 0.f)
            e = cudaMemcpyAsync(net->loss_pair + 1, net->loss_data, sizeof(float), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(net->bad_host, net->bad_index, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        *loss_host = net->loss_pair[0] + net->lambda * net->loss_pair[1];
        bad = *net->bad_host;
        if (e == cudaSuccess && bad) {
            cudaMemsetAsync(net->bad_index, 0, sizeof(int), s);
            return nn_fail(GM_EINVAL, "gm_net_train_step: an index was outside [0, count); those examples were "
                                      "zeros in this or an earlier unsynchronised step");
        }
    }
    return e == cudaSuccess ? GM_OK : nn_fail(GM_ECUDA, cudaGetErrorString(e));
}

gm_status gm_net_set_data_term(gm_net_handle net, gm_handle op, float lambda) {
    if (!net || !(lambda >= 0.f) || !std::isfinite(lambda))
        return nn_fail(GM_EINVAL, "gm_net_set_data_term: null network or lambda not finite and >= 0");
    if (lambda == 0.f) {
        net->lambda = 0.f;
        net->op = nullptr;
        return GM_OK;
    }
    gm_info inf{};
    if (!op || gm_get_info(op, &inf) != GM_OK)
        return nn_fail(GM_EINVAL, "gm_net_set_data_term: invalid operator handle");
    if (inf.precision != GM_F32 || inf.sx != net->S || inf.sy != net->S || inf.nx != net->S || inf.ny != net->S ||
        inf.nz != net->D)
        return nn_fail(GM_EINVAL, "gm_net_set_data_term: the operator must be FP32 with sx = sy = nx = ny = S "
                                  "(no padding) and nz = 16");
    if (!net->misfit) {
        const size_t nd = (size_t)net->max_batch * net->S * net->S, nm = nd * net->D;
        size_t total = 0;
        const bool ok = dev_alloc(&net->misfit, nd, &total) && dev_alloc(&net->gt, nm, &total) &&
                        dev_alloc(&net->mpred, nm, &total) && dev_alloc(&net->loss_data, 1, &total) &&
                        dev_alloc(&net->loss_data_part, kLossBlocks, &total);
        if (!ok) {
            cudaGetLastError();
            for (float **p : {&net->misfit, &net->gt, &net->mpred, &net->loss_data, &net->loss_data_part}) {
                cudaFree(*p);
                *p = nullptr;
            }
            return nn_fail(GM_ENOMEM, "gm_net_set_data_term: device allocation failed");
        }
    }
    net->op = op;
    net->lambda = lambda;
    return GM_OK;
}

gm_status gm_net_last_losses(gm_net_handle net, float *model_term, float *data_term) {
    if (!net || !model_term || !data_term) return nn_fail(GM_EINVAL, "gm_net_last_losses: null pointer");
    *model_term = net->loss_pair[0];
    *data_term = net->loss_pair[1];
    return GM_OK;
}

gm_status gm_net_get_params(gm_net_handle net, float *host, int64_t n, int which) {
    if (!net || !host || n != (int64_t)net->nparam || which < 0 || which > 3)
        return nn_fail(GM_EINVAL, "gm_net_get_params: null pointer, wrong length or which outside 0..3");
    const float *src = which == 1 ? net->gw : which == 2 ? net->m1 : which == 3 ? net->m2 : net->w;
    const cudaError_t e = cudaMemcpy(host, src, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? GM_OK : nn_fail(GM_ECUDA, cudaGetErrorString(e));
}

gm_status gm_net_set_params(gm_net_handle net, const float *host, int64_t n, int which) {
    if (!net || !host || n != (int64_t)net->nparam || which < 0 || which > 3 || which == 1)
        return nn_fail(GM_EINVAL, "gm_net_set_params: null pointer, wrong length or which not 0, 2 or 3");
    float *dst = which == 2 ? net->m1 : which == 3 ? net->m2 : net->w;
    cudaError_t e = cudaMemcpy(dst, host, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && which == 0) {
        gm::nn::k_to_bf16<<<grid1(net->nparam), 256>>>(net->w, net->wb, net->nparam);
        e = cudaDeviceSynchronize();
    }
    return e == cudaSuccess ? GM_OK : nn_fail(GM_ECUDA, cudaGetErrorString(e));
}

gm_status gm_net_get_step(gm_net_handle net, int64_t *step) {
    if (!net || !step) return nn_fail(GM_EINVAL, "gm_net_get_step: null pointer");
    *step = net->step;
    return GM_OK;
}

gm_status gm_net_set_step(gm_net_handle net, int64_t step) {
    if (!net || step < 0) return nn_fail(GM_EINVAL, "gm_net_set_step: null handle or negative step");
    net->step = step;
    return GM_OK;
}

int gm_net_last_launch_count(gm_net_handle net) { return net ? net->last_launches : 0; }

const char *gm_net_last_error(void) { return g_nn_msg; }

}  // extern "C"
