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
// Weights: FP32 master copies updated by Adam, packed after every update into two BF16 GEMM
// layouts.  Every convolution (forward, data gradient, weight gradient) is an implicit GEMM on
// the tensor cores (tcgen05.mma with FP32 accumulators in tensor memory).  The weights enter as
// BF16; the FP32 activations and gradients are gathered on the fly as two BF16 terms, v = hi + lo
// with hi = bf16(v) and lo = bf16(v - hi) (relative error below 2^-17, against 2^-9 for hi
// alone), and each product is accumulated from the terms: x w = hi w + lo w, and for the weight
// gradient x g = xhi ghi + xhi glo + xlo ghi (the lo lo term is below 2^-18 of the product).
// The element-wise steps (scaling, up-sampling, ReLU masks, loss, Adam) are plain CUDA-core kernels.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/gm_warmstart.h"
#include "gm_tcgen05.cuh"

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

// ------------------------------------------------------------------------------------------
// Convolutions as implicit GEMMs on the tensor cores (tcgen05, BF16 operands, FP32 accumulators
// in tensor memory).  One CTA of 256 threads computes a 128 x BN tile of D = A B^T over K in
// blocks of 64, two shared-memory stages deep: all threads gather the next block of A and B
// (FP32 activations / gradients as BF16 hi and lo terms, packed BF16 weights) while the tensor
// cores multiply the previous one; thread 0 issues the MMAs and commits each stage to an mbarrier.
// A stage holds A hi | A lo | B (FWD, DGRAD: the weights) or A hi | A lo | B hi | B lo (WGRAD).
//
//   FWD    rows = output positions (n, o)       cols = co   K = (tap, ci)  A = x, B = packed w
//          out[n][co][o] = b[co] + D, ReLU optional; x may be up-sampled on the fly (nearest,
//          factors 1 or 2: the gather reads the stored tensor at coordinate >> factor)
//   DGRAD  rows = input positions (n, i)        cols = ci   K = (tap, co)  A = g, B = packed w^T
//          din[n][ci][i] = D   (g at o = (i + p - tap) / s where that is an integer in range)
//   WGRAD  rows = (tap, ci), plus a row of ones  cols = co   K = positions of one chunk
//          A = x shifted by the tap, B = g;  partial dW[co][ci][tap] and, from the ones row,
//          partial db[co] of the chunk
// FWD and DGRAD launches with fewer tiles than SMs split K over gridDim.z; each CTA then writes
// its raw FP32 tile to part[z][col][row] and k_splitk_finish sums the parts in a fixed order.
enum ConvMode { FWD = 0, DGRAD = 1, WGRAD = 2 };

struct ConvGemm {
    ConvDims d;
    int M;       // GEMM rows
    int ncols;   // GEMM columns
    int kreal;   // FWD / DGRAD: taps * (channels summed); WGRAD: positions N * osz
    int kpitch;  // row length of the packed weights (multiple of 64), FWD / DGRAD
    int lg;      // log2 of the channel count that K (FWD / DGRAD) or the rows (WGRAD) run over fastest
    int chunk;   // WGRAD: positions per CTA (multiple of 64)
    int taps;
    int relu;
    int ksplit, kbper;  // FWD / DGRAD: K blocks split over gridDim.z CTAs of kbper blocks each
    int us[3];          // log2 of the nearest up-sampling (z, y, x) folded into the gathers of x
    int LD, LH, LW;     // x before up-sampling (the stored tensor); (ID, IH, IW) = (LD, LH, LW) << us
    long wait_limit;
};

constexpr int kTcThreads = 256;
constexpr int kTcBK = 64;
constexpr int kTileA = 128 * kTcBK * 2;  // bytes of one A stage

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// Two FP32 values as two BF16 terms each: *hi = {bf16(a), bf16(b)}, *lo = the BF16 roundings of
// the remainders a - bf16(a), b - bf16(b) (exact in FP32: the remainder of a rounding to fewer
// bits of the same value).
__device__ __forceinline__ void split_bf16x2(float a, float b, uint32_t *hi, uint32_t *lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    *hi = *reinterpret_cast<const uint32_t *>(&h);
    *lo = *reinterpret_cast<const uint32_t *>(&l);
}

// Bytes of one shared-memory stage of a convolution launch with BN columns.
__host__ __device__ constexpr int conv_stage_bytes(int mode, int bn) {
    return 2 * (128 * 64 * 2) + (mode == 2 ? 2 : 1) * bn * 128;
}

// q = t / s for s in {1, 2}; false unless t >= 0, s divides t and q < n
__device__ __forceinline__ bool exact_div(int t, int s, int n, int &q) {
    if (t < 0) return false;
    if (s == 2) {
        if (t & 1) return false;
        t >>= 1;
    }
    q = t;
    return t < n;
}

__device__ __forceinline__ void decode_tap(int tap, int &kz, int &ky, int &kx) {
    kz = tap / 9;
    const int r = tap - 9 * kz;
    ky = r / 3;
    kx = r - 3 * ky;
}

template <int MODE>
__global__ void __launch_bounds__(kTcThreads, 3) k_conv_tc(const float *__restrict__ act, const float *__restrict__ grad,
                                                        const __nv_bfloat16 *__restrict__ wpk,
                                                        const float *__restrict__ bias, float *__restrict__ out,
                                                        float *__restrict__ out2, ConvGemm p, int bn,
                                                        int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t bars[2];
    const ConvDims &d = p.d;
    const int t = threadIdx.x;
    const int r = t & 127;  // the GEMM row this thread gathers and, in the epilogue, stores
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * bn;
    const int stage_bytes = conv_stage_bytes(MODE, bn);
    uint32_t cols = 32;
    while (cols < (uint32_t)bn) cols <<= 1;
    if (t < 32) gm::tc::tmem_alloc(&tmem_base, cols);
    if (t == 0) {
        gm::tc::mbar_init(&bars[0], 1);
        gm::tc::mbar_init(&bars[1], 1);
    }
    gm::tc::fence_before_sync();
    __syncthreads();
    gm::tc::fence_after_sync();
    const uint32_t tmem = tmem_base;

    const int osz = d.OD * d.OH * d.OW, isz = d.ID * d.IH * d.IW;
    // FWD / DGRAD: this thread's row is a position
    int rn = -1, rz = 0, ry = 0, rx = 0, ro = 0;
    if (MODE != WGRAD) {
        const int m = m0 + r;
        if (m < p.M) {
            const int per = MODE == FWD ? osz : isz;
            const int W = MODE == FWD ? d.OW : d.IW, H = MODE == FWD ? d.OH : d.IH;
            rn = m / per;
            ro = m - rn * per;
            rx = ro % W;
            ry = (ro / W) % H;
            rz = ro / (W * H);
        }
    }
    const int q0 = MODE == WGRAD ? blockIdx.z * p.chunk : 0;
    const int kb0 = MODE == WGRAD ? 0 : blockIdx.z * p.kbper;
    const int nkb = MODE == WGRAD ? p.chunk / kTcBK : min(p.kbper, p.kpitch / kTcBK - kb0);
    const int cmask = (1 << p.lg) - 1;
    const size_t lsz = (size_t)p.LD * p.LH * p.LW;  // stored (not up-sampled) x per channel
    const uint32_t idesc = gm::tc::instr_desc_bf16(128, bn);
    bool ok = true;
    int committed = -1;  // last K block whose MMAs were committed (the same in every thread)
    // WGRAD: the first of the 8 positions this thread's warp gathers in the current K block
    // (q = linear position; sample, z, y, x), decoded once here and carried from block to block
    int wq = 0, wn = 0, wz = 0, wy = 0, wx = 0;
    if (MODE == WGRAD) {
        wq = q0 + (t >> 5) * 8;
        wn = wq / osz;
        const int o = wq - wn * osz;
        wx = o % d.OW;
        wy = (o / d.OW) % d.OH;
        wz = o / (d.OW * d.OH);
    }

    for (int it = 0; it < nkb; ++it) {
        const int kb = kb0 + it;
        const int s = it & 1;
        unsigned char *sa = smem + s * stage_bytes;  // A hi
        unsigned char *sal = sa + kTileA;             // A lo
        unsigned char *sb = sal + kTileA;             // B (hi)
        unsigned char *sbl = sb + bn * 128;           // B lo (WGRAD)
        if (it >= 2) {  // the MMAs of block it - 2 read this stage
            const bool got = gm::tc::mbar_wait(&bars[s], ((it - 2) >> 1) & 1, p.wait_limit);
            if (__syncthreads_or(!got)) {
                ok = false;
                break;
            }
        }
        // ---- A: 128 rows x 8 core columns
        if (MODE == FWD || MODE == DGRAD) {
            const int C = MODE == FWD ? d.CI : d.CO;  // channels K runs over
            const float *src = MODE == FWD ? act : grad;
            const size_t cstride = MODE == FWD ? lsz : (size_t)osz;
            const float *base = src + (size_t)(rn < 0 ? 0 : rn) * C * cstride;
            for (int kc = (t >> 7) * 4; kc < (t >> 7) * 4 + 4; ++kc) {
                const int k0 = kb * kTcBK + kc * 8;
                float v[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] = 0.f;
                if (rn >= 0 && k0 < p.kreal) {
                    if (C >= 8) {  // the 8 elements share one tap
                        const int tap = k0 >> p.lg, c0 = k0 & cmask;
                        int kz, ky, kx;
                        decode_tap(tap, kz, ky, kx);
                        int a, b, c;
                        bool in;
                        if (MODE == FWD) {
                            a = rz * d.SD + kz - d.PD;
                            b = ry * d.SH + ky - d.PH;
                            c = rx * d.SW + kx - d.PW;
                            in = a >= 0 && a < d.ID && b >= 0 && b < d.IH && c >= 0 && c < d.IW;
                        } else {
                            in = exact_div(rz + d.PD - kz, d.SD, d.OD, a) && exact_div(ry + d.PH - ky, d.SH, d.OH, b) &&
                                 exact_div(rx + d.PW - kx, d.SW, d.OW, c);
                        }
                        if (in) {
                            if (MODE == FWD) {
                                a >>= p.us[0];
                                b >>= p.us[1];
                                c >>= p.us[2];
                            }
                            const int H = MODE == FWD ? p.LH : d.OH, W = MODE == FWD ? p.LW : d.OW;
                            const float *q = base + (size_t)c0 * cstride + ((size_t)a * H + b) * W + c;
#pragma unroll
                            for (int e = 0; e < 8; ++e) v[e] = q[(size_t)e * cstride];
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int k = k0 + e;
                            if (k >= p.kreal) break;
                            const int tap = k >> p.lg, ch = k & cmask;
                            int kz, ky, kx;
                            decode_tap(tap, kz, ky, kx);
                            int a, b, c;
                            bool in;
                            if (MODE == FWD) {
                                a = rz * d.SD + kz - d.PD;
                                b = ry * d.SH + ky - d.PH;
                                c = rx * d.SW + kx - d.PW;
                                in = a >= 0 && a < d.ID && b >= 0 && b < d.IH && c >= 0 && c < d.IW;
                            } else {
                                in = exact_div(rz + d.PD - kz, d.SD, d.OD, a) &&
                                     exact_div(ry + d.PH - ky, d.SH, d.OH, b) && exact_div(rx + d.PW - kx, d.SW, d.OW, c);
                            }
                            if (in) {
                                if (MODE == FWD) {
                                    a >>= p.us[0];
                                    b >>= p.us[1];
                                    c >>= p.us[2];
                                }
                                const int H = MODE == FWD ? p.LH : d.OH, W = MODE == FWD ? p.LW : d.OW;
                                v[e] = base[(size_t)ch * cstride + ((size_t)a * H + b) * W + c];
                            }
                        }
                    }
                }
                uint4 ph, pl;
                split_bf16x2(v[0], v[1], &ph.x, &pl.x);
                split_bf16x2(v[2], v[3], &ph.y, &pl.y);
                split_bf16x2(v[4], v[5], &ph.z, &pl.z);
                split_bf16x2(v[6], v[7], &ph.w, &pl.w);
                *reinterpret_cast<uint4 *>(sa + gm::tc::tile_offset(r, kc)) = ph;
                *reinterpret_cast<uint4 *>(sal + gm::tc::tile_offset(r, kc)) = pl;
            }
        } else {
            // WGRAD: warp w fills core column w (positions 8w..8w+7 of the block) of A and B, a lane
            // whole 16-byte core-matrix rows (the row's 8 positions): A rows 4 lane .. 4 lane + 3
            // (consecutive channels of one tap when CI >= 4, so a position's bounds and offset,
            // which depend on the tap only, are computed once per tap), B rows lane, lane + 32, ...
            // Each lane stores its four A rows in a rotated order so that the 32 stores of one
            // instruction cover all eight row slots of the core matrices (four-way, not 16-way,
            // bank conflicts).
            const int warp = t >> 5, lane = t & 31;
            // the 8 positions: sample (-1 past the end), (z, y, x), offset in the sample's volume
            int smp[8], pz8[8], py8[8], px8[8], po8[8];
            {
                int q = wq, n = wn, z = wz, y = wy, x = wx;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    smp[e] = q < p.kreal ? n : -1;
                    pz8[e] = z;
                    py8[e] = y;
                    px8[e] = x;
                    po8[e] = (z * d.OH + y) * d.OW + x;
                    ++q;
                    if (++x == d.OW) {
                        x = 0;
                        if (++y == d.OH) {
                            y = 0;
                            if (++z == d.OD) {
                                z = 0;
                                ++n;
                            }
                        }
                    }
                }
            }
            const int nrow = p.taps << p.lg;
            const int rot = (lane >> 1) & 3;
            int ctap = -1, off[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) off[e] = -1;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = 4 * lane + ((r + rot) & 3), kk = m0 + row;
                float v[8];
                if (kk < nrow) {
                    const int tap = kk >> p.lg, ci = kk & cmask;
                    if (tap != ctap) {
                        ctap = tap;
                        int kz, ky, kx;
                        decode_tap(tap, kz, ky, kx);
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int aa = pz8[e] * d.SD + kz - d.PD, bb = py8[e] * d.SH + ky - d.PH,
                                      cc = px8[e] * d.SW + kx - d.PW;
                            off[e] = (smp[e] >= 0 && aa >= 0 && aa < d.ID && bb >= 0 && bb < d.IH && cc >= 0 &&
                                      cc < d.IW)
                                         ? smp[e] * d.CI * (int)lsz +
                                               ((aa >> p.us[0]) * p.LH + (bb >> p.us[1])) * p.LW + (cc >> p.us[2])
                                         : -1;
                        }
                    }
                    const int cofs = ci * (int)lsz;
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[e] = off[e] >= 0 ? act[off[e] + cofs] : 0.f;
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[e] = (kk == nrow && smp[e] >= 0) ? 1.f : 0.f;  // the ones row
                }
                uint4 h, lo;
                split_bf16x2(v[0], v[1], &h.x, &lo.x);
                split_bf16x2(v[2], v[3], &h.y, &lo.y);
                split_bf16x2(v[4], v[5], &h.z, &lo.z);
                split_bf16x2(v[6], v[7], &h.w, &lo.w);
                *reinterpret_cast<uint4 *>(sa + gm::tc::tile_offset(row, warp)) = h;
                *reinterpret_cast<uint4 *>(sal + gm::tc::tile_offset(row, warp)) = lo;
            }
            for (int row = lane; row < bn; row += 32) {  // B rows co
                const int col = n0 + row;
                float v[8];
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    v[e] = (col < p.ncols && smp[e] >= 0) ? grad[((size_t)smp[e] * d.CO + col) * osz + po8[e]] : 0.f;
                uint4 h, lo;
                split_bf16x2(v[0], v[1], &h.x, &lo.x);
                split_bf16x2(v[2], v[3], &h.y, &lo.y);
                split_bf16x2(v[4], v[5], &h.z, &lo.z);
                split_bf16x2(v[6], v[7], &h.w, &lo.w);
                *reinterpret_cast<uint4 *>(sb + gm::tc::tile_offset(row, warp)) = h;
                *reinterpret_cast<uint4 *>(sbl + gm::tc::tile_offset(row, warp)) = lo;
            }
            // the next K block's first position of this warp: kTcBK further along (x fastest, then
            // y, z, sample)
            wq += kTcBK;
            wx += kTcBK;
            while (wx >= d.OW) {
                wx -= d.OW;
                if (++wy == d.OH) {
                    wy = 0;
                    if (++wz == d.OD) {
                        wz = 0;
                        ++wn;
                    }
                }
            }
        }
        // ---- B of FWD / DGRAD: bn rows x 8 core columns of packed weights
        if (MODE != WGRAD) {
            for (int pr = t; pr < bn * 8; pr += kTcThreads) {
                const int kc = pr & 7, row = pr >> 3, col = n0 + row;
                uint4 pk = make_uint4(0, 0, 0, 0);
                if (col < p.ncols)
                    pk = *reinterpret_cast<const uint4 *>(wpk + (size_t)col * p.kpitch + kb * kTcBK + kc * 8);
                *reinterpret_cast<uint4 *>(sb + gm::tc::tile_offset(row, kc)) = pk;
            }
        }
        gm::tc::fence_smem_to_async();
        __syncthreads();
        if (t == 0) {
            gm::tc::fence_after_sync();
            const uint32_t a0 = gm::tc::smem_u32(sa), al = gm::tc::smem_u32(sal);
            const uint32_t b0 = gm::tc::smem_u32(sb), bl = gm::tc::smem_u32(sbl);
#pragma unroll
            for (int j = 0; j < kTcBK / 16; ++j) {
                const uint64_t ah = gm::tc::smem_desc(a0 + j * 256), alo = gm::tc::smem_desc(al + j * 256);
                const uint64_t bh = gm::tc::smem_desc(b0 + j * 256);
                gm::tc::mma_bf16(tmem, ah, bh, idesc, it > 0 || j > 0);  // hi x hi
                gm::tc::mma_bf16(tmem, alo, bh, idesc, true);             // lo x hi
                if (MODE == WGRAD) gm::tc::mma_bf16(tmem, ah, gm::tc::smem_desc(bl + j * 256), idesc, true);  // hi x lo
            }
            gm::tc::commit(&bars[s]);
        }
        committed = it;
    }
    if (ok) {
        const bool got = gm::tc::mbar_wait(&bars[(nkb - 1) & 1], ((nkb - 1) >> 1) & 1, p.wait_limit);
        if (__syncthreads_or(!got)) ok = false;
    }
    if (!ok) {
        if (t == 0) atomicExch(err, 1);
        // A wait gave up while MMAs may still be reading the shared-memory stages and writing this
        // block's tensor memory.  The last commit arrives only once every MMA the block issued is
        // done (a commit tracks all earlier tcgen05 operations of its thread), so wait for it once
        // more, again bounded, before the block frees its columns and exits.  If that wait gives up
        // too, the columns are freed anyway: holding them would stall the next allocation on this
        // SM without limit, and the launch has already reported the error, so its outputs are void.
        if (committed >= 0) (void)gm::tc::mbar_wait(&bars[committed & 1], (committed >> 1) & 1, p.wait_limit);
        __syncthreads();
    } else {
        gm::tc::fence_after_sync();
        const int warp = t >> 5;
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
        const int half = bn >> 1, c_begin = (warp >> 2) * half;
        const int nrow = p.taps << p.lg;
        for (int cc = c_begin; cc < c_begin + half; cc += 8) {
            float v[8];
            gm::tc::tmem_ld8(tmem + lane_base + cc, v);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int col = n0 + cc + e;
                if (col >= p.ncols) continue;
                if (MODE != WGRAD && p.ksplit > 1) {
                    if (rn < 0) continue;
                    out2[((size_t)blockIdx.z * p.ncols + col) * p.M + m0 + r] = v[e];
                } else if (MODE == FWD) {
                    if (rn < 0) continue;
                    float x = v[e] + bias[col];
                    if (p.relu) x = fmaxf(x, 0.f);
                    out[((size_t)rn * d.CO + col) * osz + ro] = x;
                } else if (MODE == DGRAD) {
                    if (rn < 0) continue;
                    out[((size_t)rn * d.CI + col) * isz + ro] = v[e];
                } else {
                    const int kk = m0 + r;
                    if (kk < nrow) {
                        const int tap = kk >> p.lg, ci = kk & cmask;
                        out[(size_t)blockIdx.z * d.CO * d.CI * p.taps + ((size_t)col * d.CI + ci) * p.taps + tap] =
                            v[e];
                    } else if (kk == nrow) {
                        out2[(size_t)blockIdx.z * d.CO + col] = v[e];
                    }
                }
            }
        }
    }
    gm::tc::fence_before_sync();
    __syncthreads();
    if (t < 32) gm::tc::tmem_free(tmem, cols);
}

// out[n][c][o] = SUM_z part[z][c][m] (z < ksplit, in order) [+ bias[c], ReLU], m = n * per + o
__global__ void k_splitk_finish(const float *__restrict__ part, int ksplit, int M, int ncols, int per,
                                const float *__restrict__ bias, int relu, float *__restrict__ out) {
    const size_t total = (size_t)M * ncols;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i / M), m = (int)(i - (size_t)c * M);
        float v = 0.f;
        for (int z = 0; z < ksplit; ++z) v += part[((size_t)z * ncols + c) * M + m];
        if (bias) v += bias[c];
        if (relu) v = fmaxf(v, 0.f);
        const int n = m / per, o = m - n * per;
        out[((size_t)n * ncols + c) * per + o] = v;
    }
}

// Packed BF16 weights of every layer: wf[co][tap * CI + ci] (FWD) and wd[ci][tap * CO + co]
// (DGRAD), rows padded with zeros to a multiple of 64 elements.
struct PackTable {
    int nl;
    int CI[12], CO[12], taps[12], kf[12], kd[12];
    long long w_off[12], f_off[12], d_off[12], cum[13];
};

__global__ void k_pack_weights(const float *__restrict__ w, __nv_bfloat16 *__restrict__ wf,
                               __nv_bfloat16 *__restrict__ wd, PackTable tb) {
    const long long total = tb.cum[tb.nl];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        int l = 0;
        while (l + 1 < tb.nl && i >= tb.cum[l + 1]) ++l;
        const long long loc = i - tb.cum[l];
        const int taps = tb.taps[l], CI = tb.CI[l], CO = tb.CO[l];
        const int tap = (int)(loc % taps), ci = (int)((loc / taps) % CI), co = (int)(loc / ((long long)taps * CI));
        const __nv_bfloat16 v = __float2bfloat16(w[tb.w_off[l] + loc]);
        wf[tb.f_off[l] + (long long)co * tb.kf[l] + (long long)tap * CI + ci] = v;
        wd[tb.d_off[l] + (long long)ci * tb.kd[l] + (long long)tap * CO + co] = v;
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

// ------------------------------------------------------------------------------------------
// Convolutions with one output channel (the network's last layer) on the CUDA cores.  The GEMM
// view of such a layer has one useful column: the tensor-core kernels would pad it to 16 and
// gather 27 x CI operand rows per position for a single product each.  Here the planes a block
// needs are read into shared memory once.  A warp task is 32 consecutive x positions (one per
// lane, so shared-memory rows are read without bank conflicts) by kDirRY rows; each input row a
// lane loads serves the up to three output rows (y taps) it touches, from registers.
// Stride 1, 3 x 3 in-plane taps with padding 1, KD in {1, 3} with padding KD / 2, input optionally
// nearest up-sampled (factor 1 or 2 per axis: the stored tensor is read at coordinate >> shift).
// Weights are the BF16 values the tensor-core kernels use; products and sums are FP32.
struct DirectConv {
    int N, CI, KD;
    int OD, OH, OW;     // output = up-sampled input size
    int LD, LH, LW;     // stored input
    int us0, us1, us2;  // up-sampling shifts
    int relu;
    int planes_per_block;  // weight gradient: (n, z) planes summed by one block
};
constexpr int kDirThreads = 256;
constexpr int kDirWarps = kDirThreads / 32;
constexpr int kDirRY = 8;         // rows per warp task
constexpr int kDirTasksMax = 16;  // forward: at most two warp tasks per warp and plane
constexpr int kDirPre = 16;       // forward: stored input values per thread prefetched for the next channel

// Shared memory of the three kernels (floats): WGRAD g plane + KD stored x planes; FWD weights +
// KD stored x planes of one channel; DGRAD weights + KD g planes.
__host__ __device__ inline size_t direct_smem_floats(int mode, const DirectConv &c) {
    const size_t plane = (size_t)c.OH * c.OW, lplane = (size_t)c.LH * c.LW;
    if (mode == WGRAD) return plane + (size_t)c.KD * lplane;
    if (mode == FWD) return (size_t)c.CI * 27 + (size_t)c.KD * lplane;
    return (size_t)c.CI * 27 + (size_t)c.KD * plane;
}

__host__ __device__ inline int dir_tasks(const DirectConv &c) {
    return ((c.OW + 31) / 32) * ((c.OH + kDirRY - 1) / kDirRY);
}

// Weight gradient, block (chunk, ci), chunk covering the (n, oz) planes [chunk * P, chunk * P + P):
//   part[chunk][ci][tap] = SUM over those planes of g(n, oz, oy, ox) x(n, ci, oz + kz - PD, oy + ky - 1,
//   ox + kx - 1) (zero outside), tap = kz * 9 + ky * 3 + kx;  with ci = 0 also bpart[chunk] = SUM of g.
__global__ void __launch_bounds__(kDirThreads) k_wgrad_co1(const float *__restrict__ x, const float *__restrict__ g,
                                                           DirectConv c, float *__restrict__ part,
                                                           float *__restrict__ bpart) {
    extern __shared__ float dsm[];
    __shared__ float red[kDirWarps][28];
    const int chunk = blockIdx.x, ci = blockIdx.y;
    const int PD = c.KD / 2, taps = c.KD * 9;
    const int plane = c.OH * c.OW, lplane = c.LH * c.LW;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int XB = (c.OW + 31) / 32, tasks = dir_tasks(c);
    float *gs = dsm;          // [OH][OW]
    float *xs = gs + plane;   // [KD][LH][LW]
    float acc[27];
#pragma unroll
    for (int t = 0; t < 27; ++t) acc[t] = 0.f;
    float gsum = 0.f;
    const int p_end = min(c.N * c.OD, (chunk + 1) * c.planes_per_block);
    for (int pl = chunk * c.planes_per_block; pl < p_end; ++pl) {
        const int n = pl / c.OD, oz = pl - n * c.OD;
        __syncthreads();  // the previous plane is no longer read
        const float *gp = g + (size_t)pl * plane;
        for (int i = threadIdx.x; i < plane; i += kDirThreads) gs[i] = gp[i];
        for (int kz = 0; kz < c.KD; ++kz) {
            const int iz = oz + kz - PD;
            const bool in = iz >= 0 && iz < c.OD;
            const float *xp = x + (((size_t)n * c.CI + ci) * c.LD + (in ? (iz >> c.us0) : 0)) * lplane;
            for (int i = threadIdx.x; i < lplane; i += kDirThreads) xs[kz * lplane + i] = in ? xp[i] : 0.f;
        }
        __syncthreads();
        for (int task = warp; task < tasks; task += kDirWarps) {
            const int xb = task % XB, y0 = (task / XB) * kDirRY;
            const int px = xb * 32 + lane;
            float gr[kDirRY];
#pragma unroll
            for (int r = 0; r < kDirRY; ++r) {
                gr[r] = (px < c.OW && y0 + r < c.OH) ? gs[(y0 + r) * c.OW + px] : 0.f;
                gsum += gr[r];
            }
#pragma unroll
            for (int kz = 0; kz < 3; ++kz) {
                if (kz < c.KD) {
                    const float *xpl = xs + kz * lplane;
#pragma unroll
                    for (int ry = 0; ry < kDirRY + 2; ++ry) {
                        const int iy = y0 + ry - 1;  // input row; output row y0 + r takes it with ky = ry - r
                        if (iy >= 0 && iy < c.OH) {
                            const float *row = xpl + (iy >> c.us1) * c.LW;
                            float v[3];
#pragma unroll
                            for (int kx = 0; kx < 3; ++kx) {
                                const int ix = px + kx - 1;
                                v[kx] = (ix >= 0 && ix < c.OW) ? row[ix >> c.us2] : 0.f;
                            }
#pragma unroll
                            for (int ky = 0; ky < 3; ++ky) {
                                const int r = ry - ky;
                                if (r >= 0 && r < kDirRY) {
#pragma unroll
                                    for (int kx = 0; kx < 3; ++kx)
                                        acc[kz * 9 + ky * 3 + kx] = fmaf(gr[r], v[kx], acc[kz * 9 + ky * 3 + kx]);
                                }
                            }
                        }
                    }
                }
            }
        }
    }
    // block sums in a fixed order: warp shuffles, then the warps in order
#pragma unroll
    for (int t = 0; t < 28; ++t) {
        float v = t < 27 ? acc[t] : gsum;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][t] = v;
    }
    __syncthreads();
    if (threadIdx.x < taps || (ci == 0 && threadIdx.x == 27)) {
        float sum = 0.f;
        for (int w = 0; w < kDirWarps; ++w) sum += red[w][threadIdx.x];
        if (threadIdx.x < taps)
            part[((size_t)chunk * c.CI + ci) * taps + threadIdx.x] = sum;
        else
            bpart[chunk] = sum;
    }
}

// Forward, block = plane (n, oz):  out(n, oz, oy, ox) = b + SUM_{ci, tap} w[ci][tap]
// x(n, ci, oz + kz - PD, oy + ky - 1, ox + kx - 1), ReLU optional.  wf: the packed FWD weights of
// the layer's one output row, element (tap, ci) at tap * CI + ci.  The next channel's stored planes
// are loaded into registers while the current one is used.
__global__ void __launch_bounds__(kDirThreads) k_fwd_co1(const float *__restrict__ x, const __nv_bfloat16 *__restrict__ wf,
                                                         const float *__restrict__ bias, DirectConv c,
                                                         float *__restrict__ out) {
    extern __shared__ float dsm[];
    const int pl = blockIdx.x;
    const int n = pl / c.OD, oz = pl - n * c.OD;
    const int PD = c.KD / 2, taps = c.KD * 9;
    const int lplane = c.LH * c.LW, nload = c.KD * lplane;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int XB = (c.OW + 31) / 32, tasks = dir_tasks(c);
    float *ws = dsm;               // [CI][27]
    float *xs = ws + c.CI * 27;    // [KD][LH][LW] of the current channel
    for (int i = threadIdx.x; i < c.CI * taps; i += kDirThreads) {
        const int ci = i / taps, tap = i - ci * taps;
        ws[ci * 27 + tap] = bf(wf[(size_t)tap * c.CI + ci]);
    }
    // element i = threadIdx.x + k * kDirThreads of a channel's KD stored planes comes from offset
    // off[k] of that channel's stored volume (-1: outside the volume or past the planes: zero)
    int off[kDirPre];
#pragma unroll
    for (int k = 0; k < kDirPre; ++k) {
        const int i = threadIdx.x + k * kDirThreads;
        const int kz = i / lplane, e = i - kz * lplane, iz = oz + kz - PD;
        off[k] = (i < nload && iz >= 0 && iz < c.OD) ? (iz >> c.us0) * lplane + e : -1;
    }
    const size_t cstride = (size_t)c.LD * lplane;
    const float *xn = x + (size_t)n * c.CI * cstride;
    float pre[kDirPre];
#pragma unroll
    for (int k = 0; k < kDirPre; ++k) pre[k] = off[k] >= 0 ? xn[off[k]] : 0.f;
    const float b0 = bias[0];
    float acc[2][kDirRY];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int r = 0; r < kDirRY; ++r) acc[q][r] = b0;
    for (int ci = 0; ci < c.CI; ++ci) {
        __syncthreads();  // the previous channel's planes are no longer read
#pragma unroll
        for (int k = 0; k < kDirPre; ++k) {
            const int i = threadIdx.x + k * kDirThreads;
            if (i < nload) xs[i] = pre[k];
        }
        __syncthreads();
        if (ci + 1 < c.CI) {
            const float *xc = xn + (size_t)(ci + 1) * cstride;
#pragma unroll
            for (int k = 0; k < kDirPre; ++k) pre[k] = off[k] >= 0 ? xc[off[k]] : 0.f;
        }
        float w[27];
#pragma unroll
        for (int t = 0; t < 27; ++t) w[t] = ws[ci * 27 + t];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int task = warp + q * kDirWarps;
            if (task < tasks) {
                const int xb = task % XB, y0 = (task / XB) * kDirRY;
                const int px = xb * 32 + lane;
#pragma unroll
                for (int kz = 0; kz < 3; ++kz) {
                    if (kz < c.KD) {
                        const float *xpl = xs + kz * lplane;
#pragma unroll
                        for (int ry = 0; ry < kDirRY + 2; ++ry) {
                            const int iy = y0 + ry - 1;
                            if (iy >= 0 && iy < c.OH) {
                                const float *row = xpl + (iy >> c.us1) * c.LW;
                                float v[3];
#pragma unroll
                                for (int kx = 0; kx < 3; ++kx) {
                                    const int ix = px + kx - 1;
                                    v[kx] = (ix >= 0 && ix < c.OW) ? row[ix >> c.us2] : 0.f;
                                }
#pragma unroll
                                for (int ky = 0; ky < 3; ++ky) {
                                    const int r = ry - ky;
                                    if (r >= 0 && r < kDirRY) {
                                        const float *wk = w + kz * 9 + ky * 3;
                                        acc[q][r] = fmaf(wk[2], v[2], fmaf(wk[1], v[1], fmaf(wk[0], v[0], acc[q][r])));
                                    }
                                }
                            }
                        }
                    }
                }
            }
        }
    }
    const size_t plane = (size_t)c.OH * c.OW;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int task = warp + q * kDirWarps;
        if (task < tasks) {
            const int xb = task % XB, y0 = (task / XB) * kDirRY;
            const int px = xb * 32 + lane;
            if (px < c.OW) {
#pragma unroll
                for (int r = 0; r < kDirRY; ++r)
                    if (y0 + r < c.OH) {
                        const float v = acc[q][r];
                        out[(size_t)pl * plane + (size_t)(y0 + r) * c.OW + px] = c.relu ? fmaxf(v, 0.f) : v;
                    }
            }
        }
    }
}

// Data gradient at the up-sampled input, block = plane (n, iz):
//   gin(n, ci, iz, iy, ix) = SUM_tap w[ci][tap] g(n, iz + PD - kz, iy + 1 - ky, ix + 1 - kx) (zero outside).
// wd: the packed DGRAD weights, element (ci, tap) at ci * kd + tap (one output channel).
__global__ void __launch_bounds__(kDirThreads) k_dgrad_co1(const float *__restrict__ g, const __nv_bfloat16 *__restrict__ wd,
                                                           int kd, DirectConv c, float *__restrict__ gin) {
    extern __shared__ float dsm[];
    const int pl = blockIdx.x;
    const int n = pl / c.OD, iz = pl - n * c.OD;
    const int PD = c.KD / 2, taps = c.KD * 9;
    const int plane = c.OH * c.OW;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int XB = (c.OW + 31) / 32, tasks = dir_tasks(c);
    float *ws = dsm;               // [CI][27]
    float *gs = ws + c.CI * 27;    // [KD][OH][OW]: the g planes oz = iz + PD - kz
    for (int i = threadIdx.x; i < c.CI * taps; i += kDirThreads) {
        const int ci = i / taps, tap = i - ci * taps;
        ws[ci * 27 + tap] = bf(wd[(size_t)ci * kd + tap]);
    }
    for (int kz = 0; kz < c.KD; ++kz) {
        const int oz = iz + PD - kz;
        const bool in = oz >= 0 && oz < c.OD;
        const float *gp = g + ((size_t)n * c.OD + (in ? oz : 0)) * plane;
        for (int i = threadIdx.x; i < plane; i += kDirThreads) gs[kz * plane + i] = in ? gp[i] : 0.f;
    }
    __syncthreads();
    for (int ci = 0; ci < c.CI; ++ci) {
        float w[27];
#pragma unroll
        for (int t = 0; t < 27; ++t) w[t] = ws[ci * 27 + t];
        float *o = gin + (((size_t)n * c.CI + ci) * c.OD + iz) * plane;
        for (int task = warp; task < tasks; task += kDirWarps) {
            const int xb = task % XB, y0 = (task / XB) * kDirRY;
            const int px = xb * 32 + lane;
            float acc[kDirRY];
#pragma unroll
            for (int r = 0; r < kDirRY; ++r) acc[r] = 0.f;
#pragma unroll
            for (int kz = 0; kz < 3; ++kz) {
                if (kz < c.KD) {
                    const float *gpl = gs + kz * plane;
#pragma unroll
                    for (int ry = 0; ry < kDirRY + 2; ++ry) {
                        // g row oy = y0 + ry - 1 reaches input row iy = oy - 1 + ky, i.e. r = ry - 2 + ky
                        const int oy = y0 + ry - 1;
                        if (oy >= 0 && oy < c.OH) {
                            const float *row = gpl + oy * c.OW;
                            float u[3];  // u[m] = g at ox = px - 1 + m, which px takes with kx = 2 - m
#pragma unroll
                            for (int m = 0; m < 3; ++m) {
                                const int ox = px - 1 + m;
                                u[m] = (ox >= 0 && ox < c.OW) ? row[ox] : 0.f;
                            }
#pragma unroll
                            for (int ky = 0; ky < 3; ++ky) {
                                const int r = ry - 2 + ky;
                                if (r >= 0 && r < kDirRY) {
                                    const float *wk = w + kz * 9 + ky * 3;
                                    acc[r] = fmaf(wk[0], u[2], fmaf(wk[1], u[1], fmaf(wk[2], u[0], acc[r])));
                                }
                            }
                        }
                    }
                }
            }
            if (px < c.OW) {
#pragma unroll
                for (int r = 0; r < kDirRY; ++r)
                    if (y0 + r < c.OH) o[(size_t)(y0 + r) * c.OW + px] = acc[r];
            }
        }
    }
}

// adjoint of nearest up-sampling: gin[c][z][y][x] = SUM of gout over its (fz, fy, fx) block
// (sizes below 2^31, which gm_net_create guarantees)
__global__ void k_upsample_bwd(const float *__restrict__ gout, float *__restrict__ gin, int NC, int D, int H, int W,
                               int fz, int fy, int fx) {
    const int tot = NC * D * H * W;
    const int OH = H * fy, OW = W * fx, OD = D * fz;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += gridDim.x * blockDim.x) {
        const int x = i % W, y = (i / W) % H, zc = i / (W * H);
        const int z = zc % D, c = zc / D;
        float s = 0.f;
        for (int a = 0; a < fz; ++a)
            for (int b = 0; b < fy; ++b) {
                const float *row = gout + ((size_t)(c * OD + z * fz + a) * OH + y * fy + b) * OW + x * fx;
                for (int e = 0; e < fx; ++e) s += row[e];
            }
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

// Adam with bias correction on the FP32 master weights (the packed BF16 copies are rebuilt after)
__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m1,
                       float *__restrict__ m2, size_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.f - b1) * gi;
        const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = v;
        const float wi = w[i] - lr * (a / c1) / (sqrtf(v / c2) + eps);
        w[i] = wi;
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
    int taps, kf, kd;        // taps; packed row lengths of the FWD and DGRAD weight layouts
    size_t f_off, d_off;     // offsets of the packed layouts
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
    __nv_bfloat16 *wf = nullptr, *wd = nullptr;  // packed BF16 weights (FWD and DGRAD layouts)
    size_t nf = 0, nd = 0;
    gm::nn::PackTable pack{};
    int *tc_err = nullptr;  // set when a tensor-core wait gives up
    std::vector<float *> x, gx, gu;  // x[l]: stored input of layer l; gx / gu: gradients before / after up-sampling
    float *kpart = nullptr;          // split-K scratch of FWD / DGRAD launches
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

constexpr int kLossBlocks = 1024;

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
    size_t off = 0, fo = 0, dof = 0;
    long long cum = 0;
    gm::nn::PackTable &tb = net->pack;
    tb.nl = (int)net->layers.size();
    for (size_t k = 0; k < net->layers.size(); ++k) {
        Layer &l = net->layers[k];
        l.w_off = off;
        off += l.nw;
        l.b_off = off;
        off += l.d.CO;
        l.taps = l.d.KD * l.d.KH * l.d.KW;
        l.kf = (l.taps * l.d.CI + 63) / 64 * 64;
        l.kd = (l.taps * l.d.CO + 63) / 64 * 64;
        l.f_off = fo;
        fo += (size_t)l.d.CO * l.kf;
        l.d_off = dof;
        dof += (size_t)l.d.CI * l.kd;
        tb.CI[k] = l.d.CI;
        tb.CO[k] = l.d.CO;
        tb.taps[k] = l.taps;
        tb.kf[k] = l.kf;
        tb.kd[k] = l.kd;
        tb.w_off[k] = (long long)l.w_off;
        tb.f_off[k] = (long long)l.f_off;
        tb.d_off[k] = (long long)l.d_off;
        tb.cum[k] = cum;
        cum += (long long)l.nw;
    }
    tb.cum[net->layers.size()] = cum;
    net->nparam = off;
    net->nf = fo;
    net->nd = dof;
}

int log2_exact(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

// The one-output-channel layers that the CUDA-core kernels take (see k_wgrad_co1): stride 1,
// "same" padding, 3 x 3 in-plane taps, at most two warp tasks per warp in the forward kernel, a
// channel's stored planes within the forward kernel's register prefetch, shared memory within the
// opt-in limit.
constexpr size_t kDirSmemMax = 200 * 1024;
constexpr int kDirPlanesPerBlock = 4;  // weight gradient: (n, z) planes per block and partial

gm::nn::DirectConv direct_view(const Layer &l, int N) {
    gm::nn::DirectConv c{};
    c.N = N;
    c.CI = l.d.CI;
    c.KD = l.d.KD;
    c.OD = l.d.OD;
    c.OH = l.d.OH;
    c.OW = l.d.OW;
    c.LD = l.in_d;
    c.LH = l.in_h;
    c.LW = l.in_w;
    c.us0 = l.up[0] == 2 ? 1 : 0;
    c.us1 = l.up[1] == 2 ? 1 : 0;
    c.us2 = l.up[2] == 2 ? 1 : 0;
    c.relu = l.relu ? 1 : 0;
    c.planes_per_block = kDirPlanesPerBlock;
    return c;
}

bool direct_ok(const Layer &l) {
    const ConvDims &d = l.d;
    if (d.CO != 1 || d.SD != 1 || d.SH != 1 || d.SW != 1 || d.KH != 3 || d.KW != 3 || d.PH != 1 || d.PW != 1)
        return false;
    if ((d.KD != 1 && d.KD != 3) || d.PD != d.KD / 2 || d.OD != d.ID || d.OH != d.IH || d.OW != d.IW) return false;
    const gm::nn::DirectConv c = direct_view(l, 1);
    if (gm::nn::dir_tasks(c) > gm::nn::kDirTasksMax) return false;
    if ((long long)c.KD * c.LH * c.LW > (long long)gm::nn::kDirPre * gm::nn::kDirThreads) return false;
    for (int mode = 0; mode < 3; ++mode)
        if (sizeof(float) * gm::nn::direct_smem_floats(mode, c) > kDirSmemMax) return false;
    return true;
}

// WGRAD split of the N * osz positions: enough chunks for about two waves of CTAs, each a
// multiple of 64 positions between 256 and 8192
int wgrad_chunk(const Layer &l, int N) {
    const long long Q = (long long)N * l.d.OD * l.d.OH * l.d.OW;
    const int mt = (l.taps * l.d.CI + 1 + 127) / 128;
    const int bn = std::min(256, (l.d.CO + 15) / 16 * 16);
    const int nt = (l.d.CO + bn - 1) / bn;
    const long long want = std::max(1, (2 * 152 + mt * nt - 1) / (mt * nt));
    long long blocks = (Q + 63) / 64;
    long long per = (blocks + want - 1) / want;
    per = std::max(4LL, std::min(128LL, per));
    return (int)(per * 64);
}

int grid1(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 4096); }

constexpr long kTcWaitLimit = 1L << 22;

// Split of the K blocks of a FWD / DGRAD launch with fewer tiles than two waves need.
void fd_split(int tiles, int nkb, int &ksplit, int &kbper) {
    ksplit = 1;
    kbper = nkb;
    if (tiles >= 152) return;
    const int want = std::min(nkb, (2 * 152 + tiles - 1) / tiles);
    if (want <= 1) return;
    kbper = (nkb + want - 1) / want;
    ksplit = (nkb + kbper - 1) / kbper;
}

// GEMM view of layer l for a batch of N in one mode (everything but pointers)
template <int MODE>
gm::nn::ConvGemm gemm_view(const Layer &l, int N, int *chunks, int *bn_out) {
    gm::nn::ConvGemm p{};
    p.d = l.d;
    p.d.N = N;
    p.taps = l.taps;
    p.relu = l.relu ? 1 : 0;
    p.wait_limit = kTcWaitLimit;
    p.ksplit = 1;
    p.LD = l.in_d;
    p.LH = l.in_h;
    p.LW = l.in_w;
    for (int a = 0; a < 3; ++a) p.us[a] = l.up[a] == 2 ? 1 : 0;
    *chunks = 1;
    if (MODE == gm::nn::FWD) {
        p.M = N * l.d.OD * l.d.OH * l.d.OW;
        p.ncols = l.d.CO;
        p.kreal = l.taps * l.d.CI;
        p.kpitch = l.kf;
        p.lg = log2_exact(l.d.CI);
    } else if (MODE == gm::nn::DGRAD) {
        p.M = N * l.d.ID * l.d.IH * l.d.IW;
        p.ncols = l.d.CI;
        p.kreal = l.taps * l.d.CO;
        p.kpitch = l.kd;
        p.lg = log2_exact(l.d.CO);
    } else {
        p.M = l.taps * l.d.CI + 1;
        p.ncols = l.d.CO;
        p.kreal = N * l.d.OD * l.d.OH * l.d.OW;
        p.lg = log2_exact(l.d.CI);
        p.chunk = wgrad_chunk(l, N);
        *chunks = (p.kreal + p.chunk - 1) / p.chunk;
    }
    const int bn = std::min(256, (p.ncols + 15) / 16 * 16);
    if (MODE != gm::nn::WGRAD) {
        const int tiles = ((p.M + 127) / 128) * ((p.ncols + bn - 1) / bn);
        fd_split(tiles, p.kpitch / 64, p.ksplit, p.kbper);
        *chunks = p.ksplit;
    }
    *bn_out = bn;
    return p;
}

// FP32 elements of split-K scratch a FWD / DGRAD launch of layer l for a batch of N needs
template <int MODE>
size_t split_scratch(const Layer &l, int N) {
    int ch = 1, bn = 16;
    const gm::nn::ConvGemm p = gemm_view<MODE>(l, N, &ch, &bn);
    return p.ksplit > 1 ? (size_t)p.ksplit * p.M * p.ncols : 0;
}

// Launches one tensor-core convolution of layer l for a batch of N (plus the split-K finish);
// returns the launches.  wpk: packed BF16 weights of the mode (FWD: [co][kf], DGRAD:
// [ci][kd]); out2: WGRAD bias partials, or the split-K scratch of FWD / DGRAD.
template <int MODE>
int launch_tc(const Layer &l, int N, const __nv_bfloat16 *wpk, const float *bias, const float *act,
              const float *grad, float *out, float *out2, int *err, cudaStream_t s) {
    int zdim = 1, bn = 16;
    const gm::nn::ConvGemm p = gemm_view<MODE>(l, N, &zdim, &bn);
    const dim3 grid((p.M + 127) / 128, (p.ncols + bn - 1) / bn, zdim);
    const size_t smem = 2 * (size_t)gm::nn::conv_stage_bytes(MODE, bn);
    gm::nn::k_conv_tc<MODE><<<grid, gm::nn::kTcThreads, smem, s>>>(act, grad, wpk, bias, out, out2, p, bn, err);
    if (MODE == gm::nn::WGRAD || p.ksplit == 1) return 1;
    const int per = MODE == gm::nn::FWD ? l.d.OD * l.d.OH * l.d.OW : l.d.ID * l.d.IH * l.d.IW;
    gm::nn::k_splitk_finish<<<grid1((size_t)p.M * p.ncols), 256, 0, s>>>(
        out2, p.ksplit, p.M, p.ncols, per, MODE == gm::nn::FWD ? bias : nullptr, MODE == gm::nn::FWD ? p.relu : 0, out);
    return 2;
}

// Weight-gradient partials of layer l for a batch of N: one per (n, output plane) on the CUDA-core
// path, one per position chunk on the tensor cores.
int wgrad_chunks(const Layer &l, int N) {
    if (direct_ok(l)) return (N * l.d.OD + kDirPlanesPerBlock - 1) / kDirPlanesPerBlock;
    const long long Q = (long long)N * l.d.OD * l.d.OH * l.d.OW;
    return (int)((Q + wgrad_chunk(l, N) - 1) / wgrad_chunk(l, N));
}

// One convolution of layer l in mode MODE: the CUDA-core kernels for a one-output-channel layer,
// else the tensor-core GEMM (launch_tc, same arguments); returns the launches made.
// The forward and data-gradient kernels give one block per plane: with fewer planes than two
// per SM (small batches) the tensor-core kernels, which tile positions, keep the GPU busier.
template <int MODE>
int launch_conv(const Layer &l, int N, const __nv_bfloat16 *wpk, const float *bias, const float *act,
                const float *grad, float *out, float *out2, int *err, cudaStream_t s) {
    const bool few_planes = MODE != gm::nn::WGRAD && (long long)N * l.d.OD < 2LL * 152;
    if (!direct_ok(l) || few_planes) return launch_tc<MODE>(l, N, wpk, bias, act, grad, out, out2, err, s);
    const gm::nn::DirectConv c = direct_view(l, N);
    const size_t smem = sizeof(float) * gm::nn::direct_smem_floats(MODE, c);
    const int planes = N * l.d.OD;
    if (MODE == gm::nn::FWD)
        gm::nn::k_fwd_co1<<<planes, gm::nn::kDirThreads, smem, s>>>(act, wpk, bias, c, out);
    else if (MODE == gm::nn::DGRAD)
        gm::nn::k_dgrad_co1<<<planes, gm::nn::kDirThreads, smem, s>>>(grad, wpk, l.kd, c, out);
    else
        gm::nn::k_wgrad_co1<<<dim3(wgrad_chunks(l, N), l.d.CI), gm::nn::kDirThreads, smem, s>>>(act, grad, c, out,
                                                                                                  out2);
    return 1;
}

cudaError_t set_tc_smem_limits() {
    cudaError_t e = cudaSuccess;
    const void *kerns[3] = {(void *)gm::nn::k_conv_tc<gm::nn::FWD>, (void *)gm::nn::k_conv_tc<gm::nn::DGRAD>,
                            (void *)gm::nn::k_conv_tc<gm::nn::WGRAD>};
    for (int mode = 0; mode < 3; ++mode)
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kerns[mode], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     2 * gm::nn::conv_stage_bytes(mode, 256));
    const void *direct[3] = {(void *)gm::nn::k_fwd_co1, (void *)gm::nn::k_dgrad_co1, (void *)gm::nn::k_wgrad_co1};
    for (const void *k : direct)
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDirSmemMax);
    return e;
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
        const Layer &l = net->layers[k];
        float *dst = (k + 1 < L) ? net->x[k + 1] : net->y;
        nl += launch_conv<gm::nn::FWD>(l, N, net->wf + l.f_off, net->w + l.b_off, net->x[k], nullptr, dst,
                                       net->kpart, net->tc_err, s);
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
        const int chunks = wgrad_chunks(l, N);
        float *dwp = net->wpart;
        float *dbp = net->wpart + (size_t)chunks * l.nw;
        launch_conv<gm::nn::WGRAD>(l, N, nullptr, nullptr, net->x[k], g, dwp, dbp, net->tc_err, s);
        gm::nn::k_sum_chunks<<<grid1(l.nw), 256, 0, s>>>(dwp, net->gw + l.w_off, l.nw, chunks);
        gm::nn::k_sum_chunks<<<grid1(l.d.CO), 256, 0, s>>>(dbp, net->gw + l.b_off, l.d.CO, chunks);
        nl += 3;
        if (k == 0) break;  // no gradient with respect to the data
        if (l.upsampled()) {
            nl += launch_conv<gm::nn::DGRAD>(l, N, net->wd + l.d_off, nullptr, nullptr, g, net->gu[k], net->kpart,
                                             net->tc_err, s);
            gm::nn::k_upsample_bwd<<<grid1(l.in_low(N)), 256, 0, s>>>(net->gu[k], net->gx[k], N * l.d.CI, l.in_d,
                                                                      l.in_h, l.in_w, l.up[0], l.up[1], l.up[2]);
            ++nl;
        } else {
            nl += launch_conv<gm::nn::DGRAD>(l, N, net->wd + l.d_off, nullptr, nullptr, g, net->gx[k], net->kpart,
                                             net->tc_err, s);
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
    cudaFree(n->wf);
    cudaFree(n->wd);
    cudaFree(n->tc_err);
    cudaFree(n->bad_index);
    if (n->bad_host) cudaFreeHost(n->bad_host);
    cudaFree(n->kpart);
    for (auto *v : {&n->x, &n->gx, &n->gu})
        for (float *p : *v) cudaFree(p);
    delete n;
}

bool dev_alloc(float **p, size_t elems, size_t *total) {
    *total += elems * sizeof(float);
    return cudaMalloc(p, elems * sizeof(float)) == cudaSuccess;
}

}  // namespace

// NVTX range around one C-ABI call.
struct NetNvtx {
    explicit NetNvtx(const char *name) { nvtxRangePushA(name); }
    ~NetNvtx() { nvtxRangePop(); }
    NetNvtx(const NetNvtx &) = delete;
    NetNvtx &operator=(const NetNvtx &) = delete;
};

extern "C" {

gm_net_handle gm_net_create(int grid, int depth, int max_batch, unsigned long long seed) {
    NetNvtx nv("gm_net_create");
    if (grid < 16 || grid > 1024 || grid % 16 || depth != 16 || max_batch < 1 ||
        (long long)max_batch * 256 * grid * grid >= (1LL << 31)) {
        nn_fail(GM_EINVAL, "gm_net_create: grid must be a multiple of 16 in [16, 1024], depth 16, "
                           "max_batch >= 1 and max_batch * 256 * grid^2 < 2^31");
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
              dev_alloc(&net->m2, P, &total) && cudaMalloc(&net->wf, 2 * net->nf) == cudaSuccess &&
              cudaMalloc(&net->wd, 2 * net->nd) == cudaSuccess && cudaMalloc(&net->tc_err, sizeof(int)) == cudaSuccess;
    net->x.assign(L, nullptr);
    net->gx.assign(L, nullptr);
    net->gu.assign(L, nullptr);
    size_t wpart = 0, kpart = 1;
    for (size_t k = 0; ok && k < L; ++k) {
        const Layer &l = net->layers[k];
        ok = dev_alloc(&net->x[k], l.in_low(B), &total) && dev_alloc(&net->gx[k], l.in_low(B), &total);
        if (ok && l.upsampled()) ok = dev_alloc(&net->gu[k], l.in_up(B), &total);
        for (int n = 1; n <= B; ++n) {  // chunk and split counts vary with the batch, not monotonically
            wpart = std::max(wpart, (size_t)wgrad_chunks(l, n) * (l.nw + l.d.CO));
            kpart = std::max(kpart, std::max(split_scratch<gm::nn::FWD>(l, n), split_scratch<gm::nn::DGRAD>(l, n)));
        }
    }
    const size_t nout = net->layers.back().out(B);
    ok = ok && dev_alloc(&net->y, nout, &total) && dev_alloc(&net->gy, nout, &total) &&
         dev_alloc(&net->target, nout, &total) && dev_alloc(&net->wpart, wpart, &total) &&
         dev_alloc(&net->kpart, kpart, &total) &&
         dev_alloc(&net->loss_part, kLossBlocks, &total) && dev_alloc(&net->loss, 1, &total) &&
         cudaMalloc(&net->bad_index, sizeof(int)) == cudaSuccess &&
         cudaMallocHost(&net->bad_host, 2 * sizeof(int)) == cudaSuccess &&
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
    if (e == cudaSuccess) e = cudaMemset(net->wf, 0, 2 * net->nf);
    if (e == cudaSuccess) e = cudaMemset(net->wd, 0, 2 * net->nd);
    if (e == cudaSuccess) e = cudaMemset(net->tc_err, 0, sizeof(int));
    if (e == cudaSuccess) e = set_tc_smem_limits();
    if (e == cudaSuccess) {
        gm::nn::k_pack_weights<<<grid1(P), 256>>>(net->w, net->wf, net->wd, net->pack);
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
    NetNvtx nv("gm_net_forward");
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
    NetNvtx nv("gm_net_train_step");
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
        gm::nn::k_adam<<<grid1(net->nparam), 256, 0, s>>>(net->w, net->gw, net->m1, net->m2, net->nparam, lr,
                                                          (float)b1, (float)b2, 1e-8f, c1, c2);
        gm::nn::k_pack_weights<<<grid1(net->nparam), 256, 0, s>>>(net->w, net->wf, net->wd, net->pack);
        nl += 2;
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
        if (e == cudaSuccess) e = cudaMemcpyAsync(net->bad_host + 1, net->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        *loss_host = net->loss_pair[0] + net->lambda * net->loss_pair[1];
        bad = *net->bad_host;
        if (e == cudaSuccess && net->bad_host[1]) {
            cudaMemsetAsync(net->tc_err, 0, sizeof(int), s);
            return nn_fail(GM_ECUDA, "gm_net_train_step: a tensor-core wait gave up; results of this or an earlier "
                                     "unsynchronised call are invalid");
        }
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
        gm::nn::k_pack_weights<<<grid1(net->nparam), 256>>>(net->w, net->wf, net->wd, net->pack);
    }
    // a copy from pageable memory may return before it lands; later work may come on any stream
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
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

gm_status gm_conv3d(int mode, int N, int CI, int CO, int ID, int IH, int IW, int KD, int stride, const float *x,
                    const float *g, const float *w, const float *b, float *out, float *bias_grad, void *stream) {
    auto pow2 = [](int v) { return v >= 1 && (v & (v - 1)) == 0; };
    if (mode < 0 || mode > 2 || N < 1 || !pow2(CI) || !pow2(CO) || CI > 4096 || CO > 4096 || ID < 1 || IH < 1 ||
        IW < 1 || (KD != 1 && KD != 3) || (stride != 1 && stride != 2) || !w || !out ||
        (mode != 1 && !x) || (mode != 0 && !g))
        return nn_fail(GM_EINVAL, "gm_conv3d: bad mode, size, channel count (powers of two), kernel depth, "
                                  "stride or null pointer");
    Layer l{};
    l.d.CI = CI;
    l.d.CO = CO;
    l.d.ID = ID;
    l.d.IH = IH;
    l.d.IW = IW;
    l.d.KD = KD;
    l.d.KH = 3;
    l.d.KW = 3;
    l.d.SD = 1;
    l.d.SH = stride;
    l.d.SW = stride;
    l.d.PD = KD / 2;
    l.d.PH = 1;
    l.d.PW = 1;
    l.d.OD = ID;
    l.d.OH = (IH - 1) / stride + 1;
    l.d.OW = (IW - 1) / stride + 1;
    l.in_d = ID;
    l.in_h = IH;
    l.in_w = IW;
    l.up[0] = l.up[1] = l.up[2] = 1;
    l.taps = KD * 9;
    l.kf = (l.taps * CI + 63) / 64 * 64;
    l.kd = (l.taps * CO + 63) / 64 * 64;
    l.nw = (size_t)CO * CI * l.taps;
    const long long rows = (long long)N * std::max(ID * IH * IW, l.d.OD * l.d.OH * l.d.OW);
    if (rows * std::max(CI, CO) > (1LL << 31) - 1 || rows > (1LL << 30))
        return nn_fail(GM_EINVAL, "gm_conv3d: tensor too large");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    gm::nn::PackTable tb{};
    tb.nl = 1;
    tb.CI[0] = CI;
    tb.CO[0] = CO;
    tb.taps[0] = l.taps;
    tb.kf[0] = l.kf;
    tb.kd[0] = l.kd;
    tb.cum[1] = (long long)l.nw;
    __nv_bfloat16 *wf = nullptr, *wd = nullptr;
    float *part = nullptr, *kpart = nullptr;
    int *err = nullptr;
    const int chunks = wgrad_chunks(l, N);
    const size_t ksz = mode == 0 ? split_scratch<gm::nn::FWD>(l, N) : mode == 1 ? split_scratch<gm::nn::DGRAD>(l, N) : 0;
    cudaError_t e = set_tc_smem_limits();
    if (e == cudaSuccess && ksz) e = cudaMalloc(&kpart, sizeof(float) * ksz);
    if (e == cudaSuccess) e = cudaMalloc(&wf, 2 * (size_t)CO * l.kf);
    if (e == cudaSuccess) e = cudaMalloc(&wd, 2 * (size_t)CI * l.kd);
    if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
    if (e == cudaSuccess && mode == 2) e = cudaMalloc(&part, sizeof(float) * (size_t)chunks * (l.nw + CO));
    if (e == cudaSuccess) e = cudaMemsetAsync(wf, 0, 2 * (size_t)CO * l.kf, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(wd, 0, 2 * (size_t)CI * l.kd, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
    int bad = 0;
    if (e == cudaSuccess) {
        gm::nn::k_pack_weights<<<grid1(l.nw), 256, 0, s>>>(w, wf, wd, tb);
        if (mode == 0) {
            float *zero = nullptr;
            if (!b) {  // a zero bias
                e = cudaMalloc(&zero, sizeof(float) * CO);
                if (e == cudaSuccess) e = cudaMemsetAsync(zero, 0, sizeof(float) * CO, s);
            }
            if (e == cudaSuccess) launch_conv<gm::nn::FWD>(l, N, wf, b ? b : zero, x, nullptr, out, kpart, err, s);
            if (zero) {
                cudaStreamSynchronize(s);
                cudaFree(zero);
            }
        } else if (mode == 1) {
            launch_conv<gm::nn::DGRAD>(l, N, wd, nullptr, nullptr, g, out, kpart, err, s);
        } else {
            launch_conv<gm::nn::WGRAD>(l, N, nullptr, nullptr, x, g, part, part + (size_t)chunks * l.nw, err, s);
            gm::nn::k_sum_chunks<<<grid1(l.nw), 256, 0, s>>>(part, out, l.nw, chunks);
            if (bias_grad)
                gm::nn::k_sum_chunks<<<grid1(CO), 256, 0, s>>>(part + (size_t)chunks * l.nw, bias_grad, CO, chunks);
        }
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    cudaFree(wf);
    cudaFree(wd);
    cudaFree(part);
    cudaFree(kpart);
    cudaFree(err);
    if (e != cudaSuccess) return nn_fail(GM_ECUDA, cudaGetErrorString(e));
    if (bad) return nn_fail(GM_ECUDA, "gm_conv3d: a tensor-core wait gave up");
    return GM_OK;
}

int gm_net_last_launch_count(gm_net_handle net) { return net ? net->last_launches : 0; }

const char *gm_net_last_error(void) { return g_nn_msg; }

}  // extern "C"
