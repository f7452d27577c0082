// gm_fast.cuh -- register-resident two-pass FFT kernels of the apply path.
//
// A transform of length N = R1 * R2 runs as two passes of straight-line DFT
// codelets in registers with one shared-memory exchange between them
// (Stockham order, natural order in and out):
//   pass 1: item j < R2 takes x[j + R2*rr] (rr < R1), runs DFT-R1 and stores its
//           outputs s < R1 in exchange row j (index n = R1*j + s);
//   pass 2: item j < R1 takes y[j + R1*rr] (rr < R2), multiplies by the twiddle
//           exp(-+2 pi i rr j / N), runs DFT-R2 and holds X[j + R1*s] (s < R2).
// Exchange rows are padded to an odd pitch so that both the row-wise stores of
// pass 1 and the column-wise loads of pass 2 hit distinct shared-memory banks.
//
// The kernels realise the steps of Eq. GrviaT / Algorithm multbttb (see apply.cu
// for the data flow); each keeps its inputs and outputs coalesced by choosing which
// of the two radices faces global memory.
#pragma once

#include "gm_common.cuh"
#include "gm_fft_codelets.cuh"

namespace gm {
namespace fast {

template <int R> struct Pitch { static constexpr int value = (R % 2) ? R : R + 1; };

// Exchange size (complex values) of one transform whose pass 1 has radix R1, rounded up to an
// odd count so that consecutive transforms start in different banks.
template <int R1, int R2> struct Ex {
    static constexpr int raw = R2 * Pitch<R1>::value;
    static constexpr int value = (raw % 2) ? raw : raw + 1;
};

// Shared-memory region of one row pair in the c2r row kernel (radices R1, R2): the two staged
// half spectra (2 (N/2 + 1) values) and, after them, the pair's exchange (Ex values) in place.
template <int R1, int R2> struct C2rRegion {
    static constexpr int staged = 2 * ((R1 * R2) / 2 + 1), ex = Ex<R1, R2>::value;
    static constexpr int value = staged > ex ? staged : ex;
};

// Asks the memory system to bring `bytes` (a multiple of 16) at a 16-byte aligned global address
// into L2; fire-and-forget, nothing waits on it.
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned int bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// L2 residency of the apply pipeline.  The spectrum and the input vector are each read once per
// product: they are loaded with an evict-first policy so that they do not push the row-FFT
// intermediates (written with evict-last) out of L2 between the kernel that writes them and the
// kernel that reads them; the reader then discards the 128-byte lines it alone owns, so dead
// intermediates are never written back to DRAM.
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ float ld_hint(const float *p, uint64_t pol) {
    float v;
    asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ double ld_hint(const double *p, uint64_t pol) {
    double v;
    asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float2 ld_hint(const float2 *p, uint64_t pol) {
    float2 v;
    asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ double2 ld_hint(const double2 *p, uint64_t pol) {
    double2 v;
    asm volatile("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ dfr ld_hint(const dfr *p, uint64_t pol) {
    dfr v;
    asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.h), "=f"(v.l) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ dfc ld_hint(const dfc *p, uint64_t pol) {
    dfc v;
    asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.h.x), "=f"(v.h.y), "=f"(v.l.x), "=f"(v.l.y)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_hint(dfc *p, dfc v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.h.x), "f"(v.h.y),
                 "f"(v.l.x), "f"(v.l.y), "l"(pol)
                 : "memory");
}
// read-only (non-coherent) load of data no kernel writes while this one runs
__device__ __forceinline__ float2 ld_nc(const float2 *p) { return __ldg(p); }
__device__ __forceinline__ double2 ld_nc(const double2 *p) { return __ldg(p); }
__device__ __forceinline__ dfc ld_nc(const dfc *p) {
    dfc v;
    asm("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.h.x), "=f"(v.h.y), "=f"(v.l.x), "=f"(v.l.y) : "l"(p));
    return v;
}
// Coherent loads cached in L2 only, for data another kernel (or another block of this one) wrote:
// the intermediates of the previous kernel in the stream, read after pdl_wait(), and the partial
// sums of other blocks.  They are volatile asm so that the compiler keeps them after pdl_wait()
// (a load through a const __restrict__ pointer may otherwise become a non-coherent load that is
// scheduled before the wait, and read the buffer before the previous kernel has written it).
__device__ __forceinline__ float2 ld_cg(const float2 *p) {
    float2 v;
    asm volatile("ld.global.cg.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ double2 ld_cg(const double2 *p) {
    double2 v;
    asm volatile("ld.global.cg.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ dfc ld_cg(const dfc *p) {
    dfc v;
    asm volatile("ld.global.cg.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.h.x), "=f"(v.h.y), "=f"(v.l.x), "=f"(v.l.y)
                 : "l"(p));
    return v;
}
// The same load predicated on ok (no access when ok is false); the value is zero then.
__device__ __forceinline__ float2 ld_cg_if(const float2 *p, bool ok) {
    float2 v = make_float2(0.f, 0.f);
    asm volatile("{ .reg .pred q; setp.ne.b32 q, %3, 0; @q ld.global.cg.v2.f32 {%0, %1}, [%2]; }"
                 : "+f"(v.x), "+f"(v.y)
                 : "l"(p), "r"((int)ok));
    return v;
}
__device__ __forceinline__ double2 ld_cg_if(const double2 *p, bool ok) {
    double2 v = make_double2(0.0, 0.0);
    asm volatile("{ .reg .pred q; setp.ne.b32 q, %3, 0; @q ld.global.cg.v2.f64 {%0, %1}, [%2]; }"
                 : "+d"(v.x), "+d"(v.y)
                 : "l"(p), "r"((int)ok));
    return v;
}
__device__ __forceinline__ dfc ld_cg_if(const dfc *p, bool ok) {
    dfc v;
    v.h = make_float2(0.f, 0.f);
    v.l = make_float2(0.f, 0.f);
    asm volatile("{ .reg .pred q; setp.ne.b32 q, %5, 0; @q ld.global.cg.v4.f32 {%0, %1, %2, %3}, [%4]; }"
                 : "+f"(v.h.x), "+f"(v.h.y), "+f"(v.l.x), "+f"(v.l.y)
                 : "l"(p), "r"((int)ok));
    return v;
}
__device__ __forceinline__ void st_hint(float2 *p, float2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void st_hint(double2 *p, double2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(p), "d"(v.x), "d"(v.y), "l"(pol)
                 : "memory");
}
// Drop the 128-byte L2 line at p (128-byte aligned) without writing it back; its contents
// become undefined.  Only for lines that no thread reads again before they are rewritten.
__device__ __forceinline__ void discard_line(const void *p) {
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

// Real even spectra (gravity, symmetric padding): the stored spectrum of layer r is the real
// E_r(kx, ky) (ky <= N/2, even in ky) of the station-centred generator, and the spectrum of the
// embedded generator is T_r = w * E_r with the separable phase
//   w(kx, ky) = exp(+2 pi i (pxl kx / NX + pyl ky / N)) = conj(twx[pxl kx mod NX]) conj(tw[pyl ky mod N]),
// tw / twx the tables exp(-2 pi i e / N).  w is the same for every layer, so the forward applies it
// once to the depth sum and the transpose applies conj(w) once to the data transform.
// Multiplies v[s] (s < R2, frequency ky = j + R1 s) by w(kx, ky), or by conj(w) when CONJ; the
// ky exponent advances by pyl R1 mod N per s (all products stay below 2^31 for N, NX <= 4096).
template <int R1, int R2, bool CONJ, typename C>
__device__ __forceinline__ void apply_phase(C (&v)[R2], const C *__restrict__ twx, int NX, int pxl, int kx,
                                            const C *tw, int N, int pyl, int j) {
    const C wx = c_conj(twx[(pxl * kx) % NX]);
    int e = (pyl * j) % N;
    const int de = (pyl * R1) % N;
#pragma unroll
    for (int s = 0; s < R2; ++s) {
        const C w = c_mul(wx, c_conj(tw[e]));
        v[s] = c_mul(v[s], CONJ ? c_conj(w) : w);
        e += de;
        if (e >= N) e -= N;
    }
}

// Index of frequency ky = j + R1 s in a real even spectrum stored for ky <= N/2 (N = R1 R2): with
// R2 even, s < R2/2 never passes N/2 and s >= R2/2 always maps to N - ky = R1 (R2 - s) - j, so
// both halves are a lane base plus a compile-time offset.
template <int R1, int R2>
__device__ __forceinline__ int even_index(int j, int s) {
    constexpr int N = R1 * R2;
    if constexpr (R2 % 2 == 0) {
        return s < R2 / 2 ? j + R1 * s : R1 * (R2 - s) - j;
    } else {
        const int ky = j + R1 * s;
        return ky <= N / 2 ? ky : N - ky;
    }
}

template <int R1, bool INV, typename C>
__device__ __forceinline__ void pass1_store(C (&v)[R1], C *ex, int j) {
    cl::Dft<R1, INV>::run(v);
    constexpr int P = Pitch<R1>::value;
#pragma unroll
    for (int s = 0; s < R1; ++s) ex[j * P + s] = v[s];
}

template <int R1, int R2, typename C>
__device__ __forceinline__ void pass2_gather(C (&v)[R2], const C *ex, int j) {
    constexpr int P = Pitch<R1>::value;
#pragma unroll
    for (int rr = 0; rr < R2; ++rr) v[rr] = ex[rr * P + j];
}

// twiddles from a table of exp(-2 pi i e / N), e < N (conjugated for the inverse): the global
// table through the read-only cache, or a shared-memory copy
template <int R1, int R2, bool INV, typename C>
__device__ __forceinline__ void pass2_twiddle_table(C (&v)[R2], const C *__restrict__ tw, int j) {
#pragma unroll
    for (int rr = 1; rr < R2; ++rr) {
        C w = tw[rr * j];
        if (INV) w = c_conj(w);
        v[rr] = c_mul(v[rr], w);
    }
}

// Copies the N-entry twiddle table to shared memory, all loads of a thread issued together.
template <int N, int THREADS, typename C>
__device__ __forceinline__ void load_table(C *dst, const C *__restrict__ src) {
    constexpr int B = (N + THREADS - 1) / THREADS;
    C tmp[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int i = threadIdx.x + b * THREADS;
        if (i < N) tmp[b] = ld_nc(src + i);
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int i = threadIdx.x + b * THREADS;
        if (i < N) dst[i] = tmp[b];
    }
}

// Per-pass twiddle layout for the pass-2 items of a transform with radices (P1, P2):
// dst[rr * P1 + j] = exp(-2 pi i rr j / N) for rr < P2, j < P1 (N = P1 P2), copied from the N-entry
// table.  Consecutive items j then read consecutive entries (no shared-memory bank conflicts,
// unlike tw[rr * j], whose stride rr sends even rr to a few banks).
template <int P1, int P2, int THREADS, typename C>
__device__ __forceinline__ void load_pass_table(C *dst, const C *__restrict__ src) {
    constexpr int N = P1 * P2, B = (N + THREADS - 1) / THREADS;
    C tmp[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int i = threadIdx.x + b * THREADS;
        if (i < N) {
            const int rr = i / P1, j = i - rr * P1;
            tmp[b] = ld_nc(src + rr * j);
        }
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int i = threadIdx.x + b * THREADS;
        if (i < N) dst[i] = tmp[b];
    }
}

// pass-2 twiddles of item j from a per-pass table (conjugated for the inverse)
template <int P1, int P2, bool INV, typename C>
__device__ __forceinline__ void pass2_twiddle_pass_table(C (&v)[P2], const C *tp, int j) {
#pragma unroll
    for (int rr = 1; rr < P2; ++rr) {
        C w = tp[rr * P1 + j];
        if (INV) w = c_conj(w);
        v[rr] = c_mul(v[rr], w);
    }
}

// The column kernels keep the per-pass twiddle tables in FP32 only: the FP64 and double-float
// kernels are bound by the FP64 pipe or by shared memory (the tables would push the 768-point
// FP64 transpose kernel past the 227 KB a block may use), so they index the N-entry table.
template <typename C> constexpr bool pass_tables() { return sizeof(C) == 8; }

// Blocks per SM the column kernels are compiled for: two for FP32 when two blocks' shared memory
// fits an SM (the register limit this sets, 128 per thread, holds the kernels without spills),
// else one (FP64 and double-float column kernels are limited to one block by shared memory).
template <typename C> constexpr int col_min_blocks(size_t smem_bytes) {
    return (sizeof(C) == 8 && smem_bytes <= 110 * 1024) ? 2 : 1;
}

// ------------------------------------------------------------------------------------------
// Real rows -> half spectra (two rows per complex transform, N = R1*R2 = N'_x).
// Block (pair group, layer) transforms rows q0 .. q0 + 2*PAIRS - 1 of `layer` of
// in[layer][row][0:row_len] and writes out[k][layer][row] (row stride out_rows), k < N/2+1.
template <typename C, typename Rin, int R1, int R2, int PAIRS, int THREADS>
__global__ void __launch_bounds__(THREADS) k_rows_r2c(const Rin *__restrict__ in, int rows, int row_len, int nlayers,
                                                      C *__restrict__ out, int out_rows, const C *__restrict__ tw) {
    constexpr int N = R1 * R2, EX = Ex<R1, R2>::value, Kx = N / 2 + 1;
    static_assert(THREADS == 32 * PAIRS && R1 <= 32 && R2 <= 32, "one warp per row pair, one item per lane");
    extern __shared__ unsigned char smem_raw[];
    C *ex = reinterpret_cast<C *>(smem_raw);
    const int q0 = blockIdx.x * 2 * PAIRS;
    const int layer = blockIdx.y;
    const uint64_t pol_in = policy_evict_first(), pol_out = policy_evict_last();
    // warp p transforms pair p on its own: both passes and the exchange stay inside the warp
    const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    pdl_wait();
    if (lane < R2) {
        const int p = wp, j = lane;
        const int qa = q0 + 2 * p;
        const bool va = qa < rows, vb = qa + 1 < rows;
        const Rin *ra = in + ((size_t)layer * rows + qa) * row_len;
        C v[R1];
#pragma unroll
        for (int rr = 0; rr < R1; ++rr) {
            const int n = j + R2 * rr;
            const bool ok = n < row_len;
            using Re = typename real_of<C>::type;
            const Re re = (ok && va) ? (Re)ld_hint(ra + n, pol_in) : Re(0);
            const Re im = (ok && vb) ? (Re)ld_hint(ra + row_len + n, pol_in) : Re(0);
            v[rr] = c_make<C>(re, im);
        }
        pass1_store<R1, false>(v, ex + p * EX, j);
    }
    __syncwarp();
    // pass 2 keeps its outputs in registers until every lane has read the exchange
    C v[R2];
    const bool act = lane < R1;
    const int p2 = wp, j2 = lane;
    if (act) {
        pass2_gather<R1, R2>(v, ex + p2 * EX, j2);
        pass2_twiddle_table<R1, R2, false>(v, tw, j2);
        cl::Dft<R2, false>::run(v);
    }
    __syncwarp();
    if (act) {
#pragma unroll
        for (int s = 0; s < R2; ++s) ex[p2 * EX + j2 + R1 * s] = v[s];  // natural order Z[k]
    }
    __syncthreads();  // the separation below reads every pair (coalesced stores across pairs)
    pdl_trigger();
    // separate the two real rows: FFT(a)[k] = (Z[k] + conj Z[-k]) / 2, FFT(b)[k] = (Z[k] - conj Z[-k]) / 2i
#pragma unroll 4
    for (int it = threadIdx.x; it < PAIRS * Kx; it += THREADS) {
        const int k = it / PAIRS, p = it - k * PAIRS;
        const int qa = q0 + 2 * p;
        if (qa >= rows) continue;
        const C a = ex[p * EX + k];
        const C b = c_conj(ex[p * EX + (k == 0 ? 0 : N - k)]);
        const C x1 = c_half(c_add(a, b));               // (Z[k] + conj Z[-k]) / 2
        const C x2 = c_half(c_mul_mi(c_sub(a, b)));     // (Z[k] - conj Z[-k]) / 2i
        C *o = out + ((size_t)k * nlayers + layer) * out_rows + qa;
        st_hint(o, x1, pol_out);
        if (qa + 1 < rows) st_hint(o + 1, x2, pol_out);
    }
}

// ------------------------------------------------------------------------------------------
// Half spectra -> real rows (two rows per complex inverse transform, N = R1*R2 = N'_x).
// X(k, layer, row) = in[k*ld_k + layer*ld_layer + row*ld_row], k < N/2+1; writes
// out[layer][row][0:row_len_out] = scale * (inverse transform)[0:row_len_out].
template <typename C, typename Rout, int R1, int R2, int PAIRS, int THREADS>
// With discard_in, every (k, layer) run of the block's 2*PAIRS rows is whole 128-byte lines
// (ld_row = 1, 128-byte aligned runs) that no other block reads: they are dropped from L2 once
// read.
__global__ void __launch_bounds__(THREADS) k_rows_c2r(const C *__restrict__ in, long long ld_k, long long ld_layer,
                                                      long long ld_row, int rows, Rout *__restrict__ out,
                                                      int row_len_out, double scale, const C *__restrict__ tw,
                                                      int discard_in) {
    constexpr int N = R1 * R2, Kx = N / 2 + 1, H = N / 2, REG = C2rRegion<R1, R2>::value;
    extern __shared__ unsigned char smem_raw[];
    // region p (REG values) holds the staged rows 2p and 2p+1 ([0, Kx) and [Kx, 2Kx)) and later the
    // exchange of pair p: only warp p reads those rows, so the two uses need no block barrier
    C *const sm = reinterpret_cast<C *>(smem_raw);  // [PAIRS][REG]
    const int q0 = blockIdx.x * 2 * PAIRS;
    const int layer = blockIdx.y;
    pdl_wait();
    {
        // staging in one round: every load of a thread is issued before its shared-memory stores
        constexpr int TOT = Kx * 2 * PAIRS, BATCH = (TOT + THREADS - 1) / THREADS;
        C tmp[BATCH];
#pragma unroll
        for (int b = 0; b < BATCH; ++b) {
            const int it = threadIdx.x + b * THREADS;
            const int k = it / (2 * PAIRS), row = it - k * 2 * PAIRS;
            const int q = q0 + row;
            tmp[b] = ld_cg_if(in + (k * ld_k + layer * ld_layer + q * ld_row), it < TOT && q < rows);
        }
#pragma unroll
        for (int b = 0; b < BATCH; ++b) {
            const int it = threadIdx.x + b * THREADS;
            if (it < TOT) {
                const int k = it / (2 * PAIRS), row = it - k * 2 * PAIRS;
                sm[(row >> 1) * REG + (row & 1) * Kx + k] = tmp[b];
            }
        }
    }
    __syncthreads();
    const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    static_assert(THREADS == 32 * PAIRS && R1 <= 32 && R2 <= 32, "one warp per row pair, one item per lane");
    constexpr int LINES = 2 * PAIRS * (int)sizeof(C) / 128;  // lines of one (k, layer) run
    if constexpr (LINES > 0) {
        if (discard_in) {
            for (int it = threadIdx.x; it < Kx * LINES; it += THREADS) {
                const int k = it / LINES, ln = it - k * LINES;
                discard_line(in + k * ld_k + layer * ld_layer + q0 + ln * (128 / (int)sizeof(C)));
            }
        }
    }
    C *const ex = sm + wp * REG;  // this warp's pair: staged rows, then exchange
    if (lane < R2) {  // warp p runs both passes of pair p
        const int j = lane;
        const C *x1r = ex, *x2r = ex + Kx;
        C v[R1];
#pragma unroll
        for (int rr = 0; rr < R1; ++rr) {
            const int n = j + R2 * rr;
            const int kk = (n <= H) ? n : N - n;
            C a = x1r[kk], b = x2r[kk];
            if (n > H) { a = c_conj(a); b = c_conj(b); }
            v[rr] = c_add(a, c_mul_i(b));  // X1 + i X2
        }
        __syncwarp(R2 >= 32 ? 0xffffffffu : ((1u << R2) - 1u));  // the pair's rows are in registers
        pass1_store<R1, true>(v, ex, j);
    }
    __syncwarp();
    pdl_trigger();
    using Re = typename real_of<C>::type;
    const Re sc = (Re)scale;
    if (lane < R1) {
        const int j = lane;
        C v[R2];
        pass2_gather<R1, R2>(v, ex, j);
        pass2_twiddle_table<R1, R2, true>(v, tw, j);
        cl::Dft<R2, true>::run(v);
        const int qa = q0 + 2 * wp;
        Rout *oa = out + ((size_t)layer * rows + qa) * row_len_out;
#pragma unroll
        for (int s = 0; s < R2; ++s) {
            const int i = j + R1 * s;
            if (i < row_len_out) {
                if (qa < rows) oa[i] = (Rout)(c_re(v[s]) * sc);
                if (qa + 1 < rows) oa[row_len_out + i] = (Rout)(c_im(v[s]) * sc);
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// Sum of the layer-group partials of COLS columns and their inverse column transform
// (N = R1*R2 = N'_y, inverse radices (R2, R1)): B[kx][j] = IFFT_y(SUM_g part[g][kx])[j], j < sy.
// Run by the whole block; ex holds COLS exchange regions of Ex<R2, R1>.
template <typename C, int R1, int R2, int COLS, int THREADS>
__device__ __forceinline__ void cols_sum_inverse(const C *__restrict__ part, int ngroups, C *__restrict__ B, int Kx,
                                                 int sy, int kx0, const C *__restrict__ tw, C *ex) {
    constexpr int IR1 = R2, IR2 = R1, N = R1 * R2, EX = Ex<IR1, IR2>::value;
    for (int it = threadIdx.x; it < COLS * IR2; it += THREADS) {
        const int c = it / IR2, j = it - c * IR2;  // pass-1 item j < IR2 takes y[j + IR2*rr], rr < IR1
        const int kx = kx0 + c;
        C v[IR1];
#pragma unroll
        for (int rr = 0; rr < IR1; ++rr) v[rr] = c_make<C>(0, 0);
        if (kx < Kx) {
            for (int g = 0; g < ngroups; ++g) {
                const C *pg = part + ((size_t)g * Kx + kx) * N + j;
                C tmp[IR1];
#pragma unroll
                for (int rr = 0; rr < IR1; ++rr) tmp[rr] = ld_cg(pg + IR2 * rr);  // written by other CTAs
#pragma unroll
                for (int rr = 0; rr < IR1; ++rr) v[rr] = c_add(v[rr], tmp[rr]);
            }
        }
        pass1_store<IR1, true>(v, ex + c * EX, j);
    }
    __syncthreads();
    for (int it = threadIdx.x; it < COLS * IR1; it += THREADS) {
        const int c = it / IR1, j = it - c * IR1;
        const int kx = kx0 + c;
        C v[IR2];
        pass2_gather<IR1, IR2>(v, ex + c * EX, j);
        pass2_twiddle_table<IR1, IR2, true>(v, tw, j);
        cl::Dft<IR2, true>::run(v);
        if (kx < Kx) {
            C *o = B + (size_t)kx * sy;
#pragma unroll
            for (int s = 0; s < IR2; ++s) {
                const int q = j + IR1 * s;
                if (q < sy) o[q] = v[s];
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// Forward column pass with the depth multiply-accumulate (N = R1*R2 = N'_y).
// Block (column group, layer group): for its COLS columns kx and layers r in the group,
// acc[kx][k] = SUM_r S[kx][r][k] * FFT_y(A[kx][r][0:ny])[k], written to part[group][kx][k].
// Pass-2 thread (c, j) owns k = j + R1*s (s < R2) for every layer, so acc stays in registers.
// The last block of a column group to finish (counted with an atomic; nothing waits) sums the
// groups' partials in group order and runs the inverse column transform into B[kx][0:sy].
// SPEC selects the spectrum form: 0 complex, 1 real even (gravity, equal padding), fixed at
// compile time so that each variant carries only its own multiply-accumulate (the unused one
// would otherwise shape the register allocation and schedule: 13 % of the FP32 kernel's time on
// the 672 x 560 grid), or 2: chosen at run time by spec_real (one kernel for both, used by the
// FP64 and double-float builds to keep their compile time down).
// Shared memory: tw [N] | tw2 [R2][R1] (per-pass layout, FP32) | exchanges.
template <typename C, int R1, int R2, int COLS, int LSTEP, int THREADS, int SPEC, int MINB>
__global__ void __launch_bounds__(THREADS, MINB)
    k_cols_fwd_mac(const C *__restrict__ A, const C *__restrict__ S, C *__restrict__ part, C *__restrict__ B,
                   unsigned int *__restrict__ counters, int Kx, int nz, int ny, int nyp, int sy,
                   int layers_per_group, int ngroups, const C *__restrict__ twg, int spec_real, int pxl, int pyl,
                   const C *__restrict__ twx) {
    const bool REAL = SPEC == 2 ? spec_real != 0 : SPEC == 1;
    constexpr int N = R1 * R2, EX = Ex<R1, R2>::value;
    static_assert(COLS * R1 <= THREADS, "one pass-2 owner per thread");
    extern __shared__ unsigned char smem_raw[];
    constexpr bool PT = pass_tables<C>();
    C *tw = reinterpret_cast<C *>(smem_raw);  // [N]
    C *tw2 = tw + N;                          // [R2][R1] (PT)
    C *ex = tw2 + (PT ? N : 0);               // [COLS*LSTEP][EX]
    __shared__ unsigned int s_last;
    const int kx0 = blockIdx.x * COLS;
    const int g = blockIdx.y;
    const int r_begin = g * layers_per_group;
    const int r_end = min(nz, r_begin + layers_per_group);
    const int t = threadIdx.x;
    const bool owner = t < COLS * R1;
    const int oc = owner ? t / R1 : 0, oj = owner ? t - oc * R1 : 0;
    const int okx = kx0 + oc;
    C acc[R2];
#pragma unroll
    for (int s = 0; s < R2; ++s) acc[s] = c_make<C>(0, 0);
    const uint64_t pol_s = policy_evict_first();
    load_table<N, THREADS>(tw, twg);
    if (PT) load_pass_table<R1, R2, THREADS>(tw2, twg);
    const int row_lines = (ny * (int)sizeof(C) + 127) / 128;  // lines of one A column (pitch nyp: whole lines)
    pdl_wait();
    for (int r = r_begin; r < r_end; r += LSTEP) {
        for (int it = t; it < COLS * LSTEP * R2; it += THREADS) {
            const int c = it / (LSTEP * R2);
            const int rem = it - c * (LSTEP * R2);
            const int l = rem / R2, j = rem - l * R2;
            const int kx = kx0 + c, rl = r + l;
            const bool valid = kx < Kx && rl < r_end;
            const C *col = A + ((size_t)(valid ? kx : 0) * nz + (valid ? rl : 0)) * nyp;
            C v[R1];
#pragma unroll
            for (int rr = 0; rr < R1; ++rr) {
                const int q = j + R2 * rr;
                v[rr] = ld_cg_if(col + q, valid && q < ny);
            }
            pass1_store<R1, false>(v, ex + (c * LSTEP + l) * EX, j);
        }
        __syncthreads();
        // every A column of this step has been read by the whole block: drop its lines
        for (int it = t; it < COLS * LSTEP * row_lines; it += THREADS) {
            const int cl_ = it / row_lines, ln = it - cl_ * row_lines;
            const int c = cl_ / LSTEP, l = cl_ - c * LSTEP;
            const int kx = kx0 + c, rl = r + l;
            if (kx < Kx && rl < r_end) discard_line(A + ((size_t)kx * nz + rl) * nyp + ln * (128 / (int)sizeof(C)));
        }
        if (owner && okx < Kx) {
#pragma unroll
            for (int l = 0; l < LSTEP; ++l) {
                const int rl = r + l;
                if (rl < r_end) {
                    C v[R2];
                    pass2_gather<R1, R2>(v, ex + (oc * LSTEP + l) * EX, oj);
                    if (PT)
                        pass2_twiddle_pass_table<R1, R2, false>(v, tw2, oj);
                    else
                        pass2_twiddle_table<R1, R2, false>(v, tw, oj);
                    cl::Dft<R2, false>::run(v);
                    if (REAL) {
                        using Rr = typename real_of<C>::type;
                        const Rr *Er = reinterpret_cast<const Rr *>(S) + ((size_t)okx * nz + rl) * (N / 2 + 1);
#pragma unroll
                        for (int s = 0; s < R2; ++s) {
                            const Rr e = ld_hint(Er + even_index<R1, R2>(oj, s), pol_s);
                            acc[s] = c_fma(v[s], e, acc[s]);
                        }
                    } else {
                        const C *Sr = S + ((size_t)okx * nz + rl) * N + oj;
#pragma unroll
                        for (int s = 0; s < R2; ++s)
                            acc[s] = c_add(acc[s], c_mul(v[s], ld_hint(Sr + R1 * s, pol_s)));
                    }
                }
            }
        }
        __syncthreads();
    }
    pdl_trigger();
    if (owner && okx < Kx) {
        if (REAL)  // the phase of the embedded generator, once for the whole depth sum
            apply_phase<R1, R2, false>(acc, twx, 2 * (Kx - 1), pxl, okx, tw, N, pyl, oj);
        C *o = part + ((size_t)g * Kx + okx) * N + oj;
#pragma unroll
        for (int s = 0; s < R2; ++s) o[R1 * s] = acc[s];
    }
    // publish the partial, then count this group in; the last group of the column group finishes it
    __threadfence();
    __syncthreads();
    if (t == 0) {
        const unsigned int prev = atomicAdd(counters + blockIdx.x, 1u);
        s_last = (prev == (unsigned int)ngroups - 1u) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (t == 0) counters[blockIdx.x] = 0u;  // ready for the next product
    static_assert(COLS * Ex<R2, R1>::value <= COLS * LSTEP * EX, "the inverse reuses the exchange buffer");
    cols_sum_inverse<C, R1, R2, COLS, THREADS>(part, ngroups, B, Kx, sy, kx0, tw, ex);
}

// ------------------------------------------------------------------------------------------
// Transpose column pass (N = R1*R2 = N'_y).  Block (column group, layer group):
// Dh = FFT_y(D1[kx][0:sy]) once (radices (R1, R2)); its pass-2 owners (c, j) keep
// Dh[j + R1*s] in registers; then for each layer the inverse transform (radices (R2, R1))
// of conj(S[kx][r]) * Dh starts from exactly those values, and A2[kx][r][q] = result[q], q < ny.
// SPEC as in k_cols_fwd_mac.  Shared memory: tw [N] | twf [R2][R1] (forward pass 2) | twi [R1][R2]
// (inverse pass 2; both FP32 only) | exchanges.
template <typename C, int R1, int R2, int COLS, int LSTEP, int THREADS, int SPEC, int MINB>
__global__ void __launch_bounds__(THREADS, MINB)
    k_cols_tr(const C *__restrict__ D1, const C *__restrict__ S, C *__restrict__ A2, int Kx, int nz, int ny, int nyp,
              int sy, int layers_per_group, const C *__restrict__ twg, int spec_real, int pxl, int pyl,
              const C *__restrict__ twx) {
    const bool REAL = SPEC == 2 ? spec_real != 0 : SPEC == 1;
    constexpr int N = R1 * R2;
    constexpr int EXF = Ex<R1, R2>::value;  // forward exchange (pass-1 radix R1)
    constexpr int EXI = Ex<R2, R1>::value;  // inverse exchange (pass-1 radix R2)
    constexpr int EXM = EXF > EXI ? EXF : EXI;
    static_assert(COLS * R1 <= THREADS, "one owner per thread");
    extern __shared__ unsigned char smem_raw[];
    constexpr bool PT = pass_tables<C>();
    C *tw = reinterpret_cast<C *>(smem_raw);  // [N]
    C *twf = tw + N;                          // [R2][R1] (PT)
    C *twi = twf + (PT ? N : 0);              // [R1][R2] (PT)
    C *ex = twi + (PT ? N : 0);               // [COLS*LSTEP][EXM]
    const int kx0 = blockIdx.x * COLS;
    const int g = blockIdx.y;
    const int r_begin = g * layers_per_group;
    const int r_end = min(nz, r_begin + layers_per_group);
    const int t = threadIdx.x;
    const bool owner = t < COLS * R1;
    const int oc = owner ? t / R1 : 0, oj = owner ? t - oc * R1 : 0;
    const int okx = kx0 + oc;
    const uint64_t pol_s = policy_evict_first(), pol_a = policy_evict_last();
    if (t < COLS * LSTEP) {
        const int c = t / LSTEP, l = t - c * LSTEP;
        const int kx = kx0 + c, rn = r_begin + l;
        if (kx < Kx && rn < r_end && !REAL)
            prefetch_l2(S + ((size_t)kx * nz + rn) * N, (unsigned int)(sizeof(C) * N));
    }
    load_table<N, THREADS>(tw, twg);
    if (PT) {
        load_pass_table<R1, R2, THREADS>(twf, twg);
        load_pass_table<R2, R1, THREADS>(twi, twg);
    }
    pdl_wait();
    // forward transform of the data columns: pass 1 items j < R2 take D1[kx][j + R2*rr]
    for (int it = t; it < COLS * R2; it += THREADS) {
        const int c = it / R2, j = it - c * R2;
        const int kx = kx0 + c;
        const C *col = D1 + (size_t)(kx < Kx ? kx : 0) * sy;
        C v[R1];
#pragma unroll
        for (int rr = 0; rr < R1; ++rr) {
            const int q = j + R2 * rr;
            v[rr] = ld_cg_if(col + q, kx < Kx && q < sy);
        }
        pass1_store<R1, false>(v, ex + c * EXM, j);
    }
    __syncthreads();
    C dh[R2];
    if (owner) {
        pass2_gather<R1, R2>(dh, ex + oc * EXM, oj);
        if (PT)
            pass2_twiddle_pass_table<R1, R2, false>(dh, twf, oj);
        else
            pass2_twiddle_table<R1, R2, false>(dh, tw, oj);
        cl::Dft<R2, false>::run(dh);
        if (REAL && okx < Kx)  // conj(T_r) Dh = E_r (conj(w) Dh): conj(w) once for all layers
            apply_phase<R1, R2, true>(dh, twx, 2 * (Kx - 1), pxl, okx, tw, N, pyl, oj);
    }
    __syncthreads();
    for (int r = r_begin; r < r_end; r += LSTEP) {
        if (t < COLS * LSTEP) {
            const int c = t / LSTEP, l = t - c * LSTEP;
            const int kx = kx0 + c, rn = r + LSTEP + l;
            if (kx < Kx && rn < r_end && !REAL)
                prefetch_l2(S + ((size_t)kx * nz + rn) * N, (unsigned int)(sizeof(C) * N));
        }
        // inverse pass 1 (radix R2) by the owners: y[oj + R1*rr] = conj(S) * Dh, rr < R2
        if (owner && okx < Kx) {
#pragma unroll
            for (int l = 0; l < LSTEP; ++l) {
                const int rl = r + l;
                if (rl < r_end) {
                    C v[R2];
                    if (REAL) {
                        using Rr = typename real_of<C>::type;
                        const Rr *Er = reinterpret_cast<const Rr *>(S) + ((size_t)okx * nz + rl) * (N / 2 + 1);
#pragma unroll
                        for (int s = 0; s < R2; ++s) {
                            const Rr e = ld_hint(Er + even_index<R1, R2>(oj, s), pol_s);
                            v[s] = c_scale(dh[s], e);
                        }
                    } else {
                        const C *Sr = S + ((size_t)okx * nz + rl) * N + oj;
#pragma unroll
                        for (int s = 0; s < R2; ++s) v[s] = c_mulc(dh[s], ld_hint(Sr + R1 * s, pol_s));
                    }
                    pass1_store<R2, true>(v, ex + (oc * LSTEP + l) * EXM, oj);
                }
            }
        }
        __syncthreads();
        // inverse pass 2 (radix R1): items j < R2, outputs q = j + R2*s (s < R1), q < ny
        for (int it = t; it < COLS * LSTEP * R2; it += THREADS) {
            const int c = it / (LSTEP * R2);
            const int rem = it - c * (LSTEP * R2);
            const int l = rem / R2, j = rem - l * R2;
            const int kx = kx0 + c, rl = r + l;
            if (kx >= Kx || rl >= r_end) continue;
            C v[R1];
            pass2_gather<R2, R1>(v, ex + (c * LSTEP + l) * EXM, j);
            if (PT)
                pass2_twiddle_pass_table<R2, R1, true>(v, twi, j);
            else
                pass2_twiddle_table<R2, R1, true>(v, tw, j);
            cl::Dft<R1, true>::run(v);
            C *o = A2 + ((size_t)kx * nz + rl) * nyp;
#pragma unroll
            for (int s = 0; s < R1; ++s) {
                const int q = j + R2 * s;
                if (q < ny) st_hint(o + q, v[s], pol_a);
            }
        }
        __syncthreads();
    }
    pdl_trigger();
}

}  // namespace fast
}  // namespace gm
