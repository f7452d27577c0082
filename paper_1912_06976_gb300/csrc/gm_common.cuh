// gm_common.cuh -- types and device helpers shared by the set-up and apply kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <set>
#include <utility>

namespace gm {

// Programmatic dependent launch: kernels launched with launch_pdl may start before the previous
// kernel on the stream has finished.  pdl_wait() blocks until that kernel has completed and its
// memory is visible (a no-op under a normal launch); a kernel calls it before its first access to
// data another kernel writes or reads.  pdl_trigger() lets the next kernel be scheduled once every
// block of this one has passed it.  The wait orders only what the compiler cannot move above it:
// data written by earlier kernels is read after it with volatile coherent loads, or through
// pointers without __restrict__ (a const __restrict__ pointer lets the compiler use non-coherent
// loads and schedule them before the wait).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

// ---- Double-float numbers: the arithmetic of GM_DF64 handles --------------------------------
// A dfr is the unevaluated sum h + l of two FP32 values with |l| <= ulp(h) / 2: a 48-bit
// significand with FP32's exponent range.  GB300 runs FP32 operations at 64 times its FP64 rate,
// so an apply with FP64 inputs, outputs and accuracy target can do its arithmetic on FP32 pairs.
// Sums use Knuth's TwoSum of the high parts and a FastTwoSum renormalisation; products use the
// exact FMA remainder of the high parts (Dekker's TwoProd with an FMA) plus the cross terms (the
// "sloppy" double-double add and multiply of Hida, Li & Bailey's QD library).  Each result is
// within a few units of 2^-47 of the exact value, measured against the operands' magnitudes,
// which is what a normwise FFT error bound needs.  The __f*_rn intrinsics keep the compiler from
// fusing or reordering the steps.
struct __align__(8) dfr {
    float h, l;
    dfr() = default;
    __host__ __device__ constexpr dfr(float hi, float lo) : h(hi), l(lo) {}
    __host__ __device__ constexpr dfr(float x) : h(x), l(0.f) {}
    __host__ __device__ constexpr dfr(int x) : h((float)x), l(0.f) {}  // small integers only (0, +-1)
    // round-to-nearest split; constant-folded for literals (the codelet coefficients)
    __host__ __device__ constexpr dfr(double x) : h((float)x), l((float)(x - (double)(float)x)) {}
    __host__ __device__ explicit constexpr operator double() const { return (double)h + (double)l; }
};
__device__ __forceinline__ dfr df_renorm(float s, float e) {  // FastTwoSum, |s| >= |e|
    const float h = __fadd_rn(s, e);
    return dfr(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ dfr operator+(dfr a, dfr b) {
    const float s = __fadd_rn(a.h, b.h);
    const float bb = __fsub_rn(s, a.h);
    float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    return df_renorm(s, e);
}
__device__ __forceinline__ dfr operator-(dfr a) { return dfr(-a.h, -a.l); }
__device__ __forceinline__ dfr operator-(dfr a, dfr b) { return a + dfr(-b.h, -b.l); }
__device__ __forceinline__ dfr operator*(dfr a, dfr b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return df_renorm(p, e);
}
__device__ __forceinline__ dfr operator*(dfr a, float c) {
    const float p = __fmul_rn(a.h, c);
    float e = __fmaf_rn(a.h, c, -p);
    e = __fmaf_rn(a.l, c, e);
    return df_renorm(p, e);
}
__device__ __forceinline__ dfr &operator+=(dfr &a, dfr b) { return a = a + b; }
__device__ __forceinline__ dfr &operator-=(dfr &a, dfr b) { return a = a - b; }

struct dfc;  // complex double-float, defined below

template <typename C> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };
template <> struct real_of<dfc> { using type = dfr; };


// Complex type of a real precision.
template <typename R> struct cpx_of;
template <> struct cpx_of<float> { using type = float2; };
template <> struct cpx_of<double> { using type = double2; };
template <> struct cpx_of<dfr> { using type = dfc; };
template <typename R> using cpx_t = typename cpx_of<R>::type;

// Element type of the caller's real vectors for an arithmetic precision (GM_DF64 takes doubles).
template <typename R> struct io_of { using type = R; };
template <> struct io_of<dfr> { using type = double; };
template <typename R> using io_t = typename io_of<R>::type;

// Complex double-float value: real and imaginary parts side by side in each half, so that one
// packed two-lane FP32 instruction (sm_100+) advances both parts of a step.  Memory order
// {re.h, im.h, re.l, im.l}.
struct __align__(16) dfc {
    float2 h, l;
};

template <typename C> __device__ __forceinline__ C c_make(typename real_of<C>::type x, typename real_of<C>::type y) {
    C c; c.x = x; c.y = y; return c;
}
template <> __device__ __forceinline__ dfc c_make<dfc>(dfr x, dfr y) {
    dfc c;
    c.h = make_float2(x.h, y.h);
    c.l = make_float2(x.l, y.l);
    return c;
}
template <typename C> __device__ __forceinline__ C c_add(C a, C b) { return c_make<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C c_sub(C a, C b) { return c_make<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C c_mul(C a, C b) {
    return c_make<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C c_mulc(C a, C b) {
    return c_make<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> __device__ __forceinline__ C c_conj(C a) { return c_make<C>(a.x, -a.y); }
template <typename C> __device__ __forceinline__ C c_mul_i(C a) { return c_make<C>(-a.y, a.x); }
template <typename C> __device__ __forceinline__ C c_mul_mi(C a) { return c_make<C>(a.y, -a.x); }
template <typename C> __device__ __forceinline__ C c_half(C a) { return c_make<C>(a.x * 0.5f, a.y * 0.5f); }
template <typename C> __device__ __forceinline__ typename real_of<C>::type c_re(C a) { return a.x; }
template <typename C> __device__ __forceinline__ typename real_of<C>::type c_im(C a) { return a.y; }
// a * e for a real e, and acc + a * e (one rounding per part)
__device__ __forceinline__ float2 c_scale(float2 a, float e) { return make_float2(a.x * e, a.y * e); }
__device__ __forceinline__ double2 c_scale(double2 a, double e) { return make_double2(a.x * e, a.y * e); }
__device__ __forceinline__ float2 c_fma(float2 a, float e, float2 acc) {
    return make_float2(fmaf(a.x, e, acc.x), fmaf(a.y, e, acc.y));
}
__device__ __forceinline__ double2 c_fma(double2 a, double e, double2 acc) {
    return make_double2(fma(a.x, e, acc.x), fma(a.y, e, acc.y));
}

// ---- packed double-float complex arithmetic (the overloads above for dfc) -------------------
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f, -1.f), a); }
__device__ __forceinline__ dfc dfc_of(float2 h, float2 l) {
    dfc c;
    c.h = h;
    c.l = l;
    return c;
}
// FastTwoSum of s + e in each lane (|s| >= |e| or s == 0)
__device__ __forceinline__ dfc dfc_renorm(float2 s, float2 e) {
    const float2 h = __fadd2_rn(s, e);
    return dfc_of(h, f2_sub(e, f2_sub(h, s)));
}
__device__ __forceinline__ dfc c_add(dfc a, dfc b) {  // TwoSum of the high parts, low parts added
    const float2 s = __fadd2_rn(a.h, b.h);
    const float2 bb = f2_sub(s, a.h);
    float2 e = __fadd2_rn(f2_sub(a.h, f2_sub(s, bb)), f2_sub(b.h, bb));
    e = __fadd2_rn(e, __fadd2_rn(a.l, b.l));
    return dfc_renorm(s, e);
}
__device__ __forceinline__ dfc c_sub(dfc a, dfc b) {  // TwoDiff of the high parts
    const float2 s = f2_sub(a.h, b.h);
    const float2 bb = f2_sub(s, a.h);
    float2 e = f2_sub(f2_sub(a.h, f2_sub(s, bb)), __fadd2_rn(b.h, bb));
    e = __fadd2_rn(e, f2_sub(a.l, b.l));
    return dfc_renorm(s, e);
}
__device__ __forceinline__ dfc c_neg(dfc a) { return dfc_of(f2(-a.h.x, -a.h.y), f2(-a.l.x, -a.l.y)); }
__device__ __forceinline__ dfc c_conj(dfc a) { return dfc_of(f2(a.h.x, -a.h.y), f2(a.l.x, -a.l.y)); }
__device__ __forceinline__ dfc c_mul_i(dfc a) { return dfc_of(f2(-a.h.y, a.h.x), f2(-a.l.y, a.l.x)); }
__device__ __forceinline__ dfc c_mul_mi(dfc a) { return dfc_of(f2(a.h.y, -a.h.x), f2(a.l.y, -a.l.x)); }
__device__ __forceinline__ dfc c_half(dfc a) {
    return dfc_of(__fmul2_rn(a.h, f2(0.5f, 0.5f)), __fmul2_rn(a.l, f2(0.5f, 0.5f)));
}
__device__ __forceinline__ dfr c_re(dfc a) { return dfr(a.h.x, a.l.x); }
__device__ __forceinline__ dfr c_im(dfc a) { return dfr(a.h.y, a.l.y); }
// lane-wise product with the double-float multiplier mh + ml of each lane
__device__ __forceinline__ dfc c_mul_lanes(dfc a, float2 mh, float2 ml) {
    const float2 pn = __fmul2_rn(a.h, f2(-mh.x, -mh.y));  // -p, p = a.h * mh rounded
    float2 e = __ffma2_rn(a.h, mh, pn);                   // exact remainder of a.h * mh
    e = __ffma2_rn(a.h, ml, e);
    e = __ffma2_rn(a.l, mh, e);
    const float2 h = f2_sub(e, pn);                       // p + e
    return dfc_of(h, f2_sub(e, __fadd2_rn(h, pn)));       // e - (h - p)
}
__device__ __forceinline__ dfc c_scale(dfc a, dfr e) { return c_mul_lanes(a, f2(e.h, e.h), f2(e.l, e.l)); }
__device__ __forceinline__ dfc c_fma(dfc a, dfr e, dfc acc) { return c_add(acc, c_scale(a, e)); }
__device__ __forceinline__ dfc c_mul(dfc a, dfc b) {  // (a.x b.x - a.y b.y, a.y b.x + a.x b.y)
    return c_add(c_mul_lanes(a, f2(b.h.x, b.h.x), f2(b.l.x, b.l.x)),
                 c_mul_lanes(c_mul_i(a), f2(b.h.y, b.h.y), f2(b.l.y, b.l.y)));
}
__device__ __forceinline__ dfc c_mulc(dfc a, dfc b) { return c_mul(a, c_conj(b)); }

// codelet helpers for dfc (the float2 / double2 forms are next to the codelets; argument-
// dependent lookup finds these from inside the codelets)
__device__ __forceinline__ dfc cx_add(dfc a, dfc b) { return c_add(a, b); }
__device__ __forceinline__ dfc cx_sub(dfc a, dfc b) { return c_sub(a, b); }
__device__ __forceinline__ dfc cx_neg(dfc a) { return c_neg(a); }
__device__ __forceinline__ dfc cx_mul_i(dfc a) { return c_mul_i(a); }
__device__ __forceinline__ dfc cx_mul_mi(dfc a) { return c_mul_mi(a); }
__device__ __forceinline__ dfc cx_scale(dfc a, dfr c) { return c_scale(a, c); }
__device__ __forceinline__ dfc cx_fma(dfc t, dfr c, dfc acc) { return c_fma(t, c, acc); }
// a (c + i s)
__device__ __forceinline__ dfc cx_rot(dfc a, dfr c, dfr s) { return c_add(c_scale(a, c), c_scale(c_mul_i(a), s)); }
// (x + i y)(c + i s) with |c| = |s|: mode 1 -> ((x - y) c, (x + y) s), mode 0 -> ((x + y) c, (x - y) s)
__device__ __forceinline__ dfc cx_rot_diag(dfc a, dfr c, dfr s, int mode) {
    const dfc xx = dfc_of(f2(a.h.x, a.h.x), f2(a.l.x, a.l.x));
    const dfc yy = mode ? dfc_of(f2(-a.h.y, a.h.y), f2(-a.l.y, a.l.y)) : dfc_of(f2(a.h.y, -a.h.y), f2(a.l.y, -a.l.y));
    return c_mul_lanes(c_add(xx, yy), f2(c.h, s.h), f2(c.l, s.l));
}
// A + sign i B and A - sign i B with sign = +-1 (a literal, so the branch folds)
__device__ __forceinline__ dfc cx_addi(dfc A, dfc B, dfr sign) { return c_add(A, sign.h > 0.f ? c_mul_i(B) : c_mul_mi(B)); }
__device__ __forceinline__ dfc cx_subi(dfc A, dfc B, dfr sign) { return c_add(A, sign.h > 0.f ? c_mul_mi(B) : c_mul_i(B)); }

// Opts a kernel into more than the default 48 KB of dynamic shared memory when needed, once
// per (kernel, device, size) so that launches do not pay for the attribute call.
template <typename K>
inline cudaError_t allow_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    static std::mutex mu;
    static std::set<std::pair<std::pair<const void *, int>, size_t>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const auto key = std::make_pair(std::make_pair((const void *)kernel, dev), bytes);
    std::lock_guard<std::mutex> lk(mu);
    if (done.count(key)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done.insert(key);
    return e;
}

// Number of SMs of the current device (queried once per device).
inline int sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (!cache[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 148;
        cache[dev] = n;
    }
    return cache[dev];
}

// Mixed-radix plan of one FFT length: the radices of its passes (product = N)
// and a table of the N roots exp(-2 pi i e / N), e < N, in the kernel's precision.
constexpr int kMaxPasses = 16;
struct FftDesc {
    int N;
    int npass;
    int radix[kMaxPasses];
    const void *tw;
};

// Geometry of a plan as the kernels see it.
struct Geo {
    int sx, sy, nz, nx, ny;     // stations, layers, padded cells
    int pxl, pyl;               // left padding
    int NPx, NPy, Kx;           // FFT lengths, kept x-columns N'_x/2+1
    int nyp;                    // ny rounded up to even: column pitch of the [kx][r][q] intermediates
};

// Batched in-place-ish Stockham autosort FFT on shared memory, all threads of
// the block cooperating.  nb transforms of length d.N live at buf0 + t*ld
// (t < nb); buf1 is scratch of the same shape.  Each pass of radix R maps
// input j + rr*(N/R) to output (j / Ns)*Ns*R + (j mod Ns) + s*Ns after the
// twiddle W_{Ns R}^{rr (j mod Ns)} and an R-point DFT (Ns = product of the
// earlier radices), so the result comes out in natural order.  Returns the
// buffer that holds the result.  inverse = unnormalised inverse transform.
// The caller synchronises the block before the call; the call ends synchronised.
template <typename C>
__device__ C *fft_block(C *buf0, C *buf1, int nb, int ld, const FftDesc &d, bool inverse) {
    const C *tw = reinterpret_cast<const C *>(d.tw);
    const int N = d.N;
    C *src = buf0, *dst = buf1;
    int Ns = 1;
    for (int ps = 0; ps < d.npass; ++ps) {
        const int R = d.radix[ps];
        const int M = N / R;
        const int step = N / (Ns * R);
        for (int item = threadIdx.x; item < nb * M; item += blockDim.x) {
            const int t = item / M;
            const int j = item - t * M;
            const int k = j % Ns;
            C v[8], o[8];
#pragma unroll
            for (int rr = 0; rr < 8; ++rr)
                if (rr < R) v[rr] = src[t * ld + j + rr * M];
#pragma unroll
            for (int rr = 1; rr < 8; ++rr)
                if (rr < R) {
                    C w = tw[(rr * k * step) % N];
                    if (inverse) w.y = -w.y;
                    v[rr] = c_mul(v[rr], w);
                }
#pragma unroll
            for (int s = 0; s < 8; ++s)
                if (s < R) {
                    C acc = v[0];
#pragma unroll
                    for (int rr = 1; rr < 8; ++rr)
                        if (rr < R) {
                            C w = tw[((rr * s) % R) * M];
                            if (inverse) w.y = -w.y;
                            acc = c_add(acc, c_mul(v[rr], w));
                        }
                    o[s] = acc;
                }
            const int base = (j / Ns) * Ns * R + k;
#pragma unroll
            for (int s = 0; s < 8; ++s)
                if (s < R) dst[t * ld + base + s * Ns] = o[s];
        }
        __syncthreads();
        C *tmp = src; src = dst; dst = tmp;
        Ns *= R;
    }
    return src;
}

}  // namespace gm
