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
// block of this one has passed it.
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

template <typename C> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };


// Complex type of a real precision.
template <typename R> struct cpx_of;
template <> struct cpx_of<float> { using type = float2; };
template <> struct cpx_of<double> { using type = double2; };
template <typename R> using cpx_t = typename cpx_of<R>::type;

template <typename C> __device__ __forceinline__ C c_make(decltype(C::x) x, decltype(C::x) y) {
    C c; c.x = x; c.y = y; return c;
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
