// cgls.cu -- Tikhonov-regularised CGLS with every step on the device.
//
// Solves min ||G x - d||^2 + alpha^2 ||x||^2 with the conjugate-gradient method
// on the normal equations (G^T G + alpha^2 I) x = G^T d, in its least-squares
// form (CGLS): per iteration one forward and one transpose product of the
// fast operator (the use the paper's conclusion names for the transpose
// product, Sec. 7) plus the vector updates below.  Scalars (gamma, delta, the
// step lengths) live in device memory, dot products are accumulated in FP64
// with a fixed two-stage reduction (bit-reproducible), and no iteration waits
// for the host.  The second stage of each reduction and the scalar update that
// follows it run in the last block of the reduction kernel to arrive, so an
// iteration takes four vector kernels besides the two products.
//
//   r = d - G x0;  s = G^T r - alpha^2 x0;  p = s;  gamma = ||s||^2
//   repeat: q = G p;  delta = ||q||^2 + alpha^2 ||p||^2;  a = gamma / delta
//           x += a p;  r -= a q;  s = G^T r - alpha^2 x
//           gamma' = ||s||^2;  b = gamma' / gamma;  gamma = gamma';  p = s + b p
//
// Once ||s|| has fallen to rounding level (||s|| <= 64 eps ||s_0||, eps of the vector
// precision) the iterate is the regularised solution to working accuracy; further steps would
// only act on rounding noise (the FFT transpose is G^T to rounding, not exactly), so the
// remaining iterations keep x and r unchanged.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "gm_plan.h"

namespace gm {

constexpr int kRedBlocks = 512;
constexpr int kRedThreads = 256;

// scalar slots (S_ARRIVE holds the arrival count of the reduction blocks, as an unsigned int)
enum { S_GAMMA = 0, S_A = 1, S_B = 2, S_ALPHA2 = 3, S_THRESH = 4, S_DONE = 5, S_ARRIVE = 6, S_COUNT = 8 };

__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    return v;
}

// Partial sums written by other blocks of the same launch, read through L2 (not L1).
__device__ double sum_parts(const double *part, double *sh) {
    double v = 0;
    for (int i = threadIdx.x; i < kRedBlocks; i += blockDim.x) v += __ldcg(part + i);
    return block_sum(v, sh);
}

// The reductions of an iteration with their scalar step fused in: every block reduces its share
// of SUM a^2 and SUM b^2 into part[], and the last block to arrive (an atomic count; nothing
// waits) sums the parts in block order and updates the scalars.  MODE
//   0 step length:  a = q, b = p;  a_step = gamma / (||q||^2 + alpha^2 ||p||^2), 0 once converged
//   1 beta:         a = s after s -= alpha^2 x, b = r;  beta = ||s||^2 / gamma, gamma = ||s||^2,
//                   resid[k] = ||r||
//   2 init:         a = s after s -= alpha^2 x and p = s, b = r;  gamma = ||s||^2, resid[0] = ||r||
template <typename R, int MODE>
__global__ void k_reduce_step(R *a, size_t na, const R *b, size_t nb, const R *x, R *pv, R a2, double *part,
                              double *sc, double *resid, int k, double alpha2, double tol2) {
    pdl_wait();
    pdl_trigger();
    __shared__ double sh[32];
    __shared__ unsigned int s_last;
    double sa = 0, sb = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < na; i += (size_t)gridDim.x * blockDim.x) {
        R v = a[i];
        if (MODE != 0) {
            v = v - a2 * x[i];
            a[i] = v;
            if (MODE == 2) pv[i] = v;
        }
        sa += (double)v * (double)v;
    }
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nb; i += (size_t)gridDim.x * blockDim.x)
        sb += (double)b[i] * (double)b[i];
    sa = block_sum(sa, sh);
    sb = block_sum(sb, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = sa;
        part[kRedBlocks + blockIdx.x] = sb;
    }
    __threadfence();
    __syncthreads();
    unsigned int *arrive = reinterpret_cast<unsigned int *>(sc + S_ARRIVE);
    if (threadIdx.x == 0) s_last = (atomicAdd(arrive, 1u) == gridDim.x - 1u) ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const double A = sum_parts(part, sh);
    const double B = sum_parts(part + kRedBlocks, sh);
    if (threadIdx.x == 0) {
        *arrive = 0u;  // ready for the next reduction
        if (MODE == 0) {
            if (sc[S_GAMMA] <= sc[S_THRESH]) sc[S_DONE] = 1.0;
            const double delta = A + sc[S_ALPHA2] * B;
            sc[S_A] = (sc[S_DONE] == 0.0 && delta > 0) ? sc[S_GAMMA] / delta : 0.0;
        } else if (MODE == 1) {
            const double g = sc[S_GAMMA];
            sc[S_B] = (sc[S_DONE] == 0.0 && g > 0) ? A / g : 0.0;
            sc[S_GAMMA] = A;
            resid[k] = sqrt(B);
        } else {
            sc[S_GAMMA] = A;
            sc[S_ALPHA2] = alpha2;
            sc[S_THRESH] = tol2 * A;
            sc[S_DONE] = (A > 0) ? 0.0 : 1.0;
            resid[0] = sqrt(B);
        }
    }
}

// Convergence threshold on ||s||^2 / ||s_0||^2 for vectors of type R.
// squared freeze threshold: 64 units of the apply arithmetic's precision (double-float pairs
// carry a 48-bit significand, 2^-47 apart)
inline double cgls_tol2(int precision) {
    const double eps = precision == GM_F64    ? 2.220446049250313e-16
                       : precision == GM_DF64 ? 7.105427357601002e-15
                                              : 1.1920928955078125e-07;
    return (64.0 * eps) * (64.0 * eps);
}

// r = d - r (r holds G x0 on entry)
template <typename R>
__global__ void k_residual0(const R *d, R *r, size_t m) {
    pdl_wait();
    pdl_trigger();
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x)
        r[i] = d[i] - r[i];
}

// x += a p (i < n); r -= a q (i < m)
template <typename R>
__global__ void k_update_xr(R *x, const R *p, size_t n, R *r,
                            const R *q, size_t m, const double *sc) {
    pdl_wait();
    pdl_trigger();
    const R a = (R)sc[S_A];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        x[i] += a * p[i];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x)
        r[i] -= a * q[i];
}

// p = s + b p
template <typename R>
__global__ void k_update_p(R *p, const R *s, size_t n, const double *sc) {
    pdl_wait();
    pdl_trigger();
    const R b = (R)sc[S_B];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p[i] = s[i] + b * p[i];
}

template <typename R>
static cudaError_t cgls_t(gm_plan *p, const R *d, const R *x0, R *x, double alpha, int iters, double *resid_host,
                          cudaStream_t st, int *nl) {
    const size_t n = (size_t)p->geo.nx * p->geo.ny * p->geo.nz, m = (size_t)p->geo.sx * p->geo.sy;
    const size_t vec = sizeof(R) * (2 * n + 2 * m);
    const size_t need = vec + sizeof(double) * (2 * kRedBlocks + S_COUNT + (size_t)iters + 1) + 256;
    if (need > p->cgls_bytes) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        cudaFree(p->cgls_buf);
        p->cgls_buf = nullptr;
        p->cgls_bytes = 0;
        e = cudaMalloc(&p->cgls_buf, need);
        if (e != cudaSuccess) return e;
        p->cgls_bytes = need;
    }
    char *base = static_cast<char *>(p->cgls_buf);
    R *s = reinterpret_cast<R *>(base);
    R *pv = s + n;
    R *r = pv + n;
    R *q = r + m;
    double *part = reinterpret_cast<double *>(base + ((sizeof(R) * (2 * n + 2 * m) + 255) / 256) * 256);
    double *sc = part + 2 * kRedBlocks;
    double *resid = sc + S_COUNT;
    int launches = 0, k = 0;
    cudaError_t e = cudaSuccess;
    const int vb = kRedBlocks, vt = kRedThreads;
#define CG_TRY(x)                                  \
    do {                                           \
        e = (x);                                   \
        if (e != cudaSuccess) goto out;            \
    } while (0)
    CG_TRY(cudaMemsetAsync(sc, 0, sizeof(double) * S_COUNT, st));  // the arrival count starts at zero
    if (x0 && x0 != x) CG_TRY(cudaMemcpyAsync(x, x0, sizeof(R) * n, cudaMemcpyDeviceToDevice, st));
    if (!x0) CG_TRY(cudaMemsetAsync(x, 0, sizeof(R) * n, st));
    {
        int l = 0;
        CG_TRY(launch_forward(p, x, r, st, &l));  // r = G x0
        launches += l;
    }
    launch_pdl(k_residual0<R>, dim3(vb), dim3(vt), 0, st, d, r, m);
    {
        int l = 0;
        CG_TRY(launch_transpose(p, r, s, st, &l));  // s = G^T r
        launches += l;
    }
    launch_pdl(k_reduce_step<R, 2>, dim3(vb), dim3(vt), 0, st, s, n, (const R *)r, m, (const R *)x, pv,
               (R)(alpha * alpha), part, sc, resid, 0, alpha * alpha, cgls_tol2(p->precision));
    launches += 2;
    for (k = 1; k <= iters; ++k) {
        int l = 0;
        CG_TRY(launch_forward(p, pv, q, st, &l));  // q = G p
        launches += l;
        launch_pdl(k_reduce_step<R, 0>, dim3(vb), dim3(vt), 0, st, q, m, (const R *)pv, n, (const R *)nullptr,
                   (R *)nullptr, (R)0, part, sc, resid, k, 0.0, 0.0);
        launch_pdl(k_update_xr<R>, dim3(vb), dim3(vt), 0, st, x, pv, n, r, q, m, sc);
        CG_TRY(launch_transpose(p, r, s, st, &l));  // s = G^T r
        launches += l;
        launch_pdl(k_reduce_step<R, 1>, dim3(vb), dim3(vt), 0, st, s, n, (const R *)r, m, (const R *)x,
                   (R *)nullptr, (R)(alpha * alpha), part, sc, resid, k, 0.0, 0.0);
        launch_pdl(k_update_p<R>, dim3(vb), dim3(vt), 0, st, pv, s, n, sc);
        launches += 4;
        CG_TRY(cudaGetLastError());
    }
    CG_TRY(cudaGetLastError());
    if (resid_host) {
        CG_TRY(cudaMemcpyAsync(resid_host, resid, sizeof(double) * (iters + 1), cudaMemcpyDeviceToHost, st));
        CG_TRY(cudaStreamSynchronize(st));
    }
out:
#undef CG_TRY
    *nl = launches;
    return e;
}

// ---------------------------------------------------------------------------------------------
// Allocation-free CGLS (gm_cgls_noalloc).  Same iteration and kernels as cgls_t above, but its
// scratch (four vectors, the reduction partials, the scalars and the residual history) lives in
// one fixed file-scope device array instead of memory the handle allocates on first use.  The
// array is shared by every call in the process: its contents persist between calls and calls
// that overlap on the GPU would race on it.
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB on every GPU that loads the library
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mutex;
static void *g_noalloc_ptr[kMaxDevices] = {};

size_t noalloc_scratch_bytes() { return kNoAllocScratchBytes; }

// Device address of the array on the current device, looked up once per device (the host-side
// name of a __device__ variable is not a device address).
static cudaError_t noalloc_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = ptr;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

size_t noalloc_cgls_need(const gm_plan *p, int iters) {
    const size_t n = (size_t)p->geo.nx * p->geo.ny * p->geo.nz, m = (size_t)p->geo.sx * p->geo.sy;
    const size_t el = p->precision == GM_F32 ? sizeof(float) : sizeof(double);
    return ((el * (2 * n + 2 * m) + 255) / 256) * 256 + sizeof(double) * (2 * kRedBlocks + S_COUNT + (size_t)iters + 1);
}

template <typename R>
static cudaError_t cgls_noalloc_t(gm_plan *p, const R *d, const R *x0, R *x, double alpha, int iters,
                                  double *resid_host, cudaStream_t st, int *nl) {
    const size_t n = (size_t)p->geo.nx * p->geo.ny * p->geo.nz, m = (size_t)p->geo.sx * p->geo.sy;
    void *scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    if (e != cudaSuccess) return e;
    char *base = static_cast<char *>(scratch);
    R *s = reinterpret_cast<R *>(base);
    R *pv = s + n;
    R *r = pv + n;
    R *q = r + m;
    double *part = reinterpret_cast<double *>(base + ((sizeof(R) * (2 * n + 2 * m) + 255) / 256) * 256);
    double *sc = part + 2 * kRedBlocks;
    double *resid = sc + S_COUNT;
    int launches = 0, k = 0;
    const int vb = kRedBlocks, vt = kRedThreads;
#define NA_TRY(x)                                  \
    do {                                           \
        e = (x);                                   \
        if (e != cudaSuccess) goto out;            \
    } while (0)
    // the array keeps the previous call's values: start the scalars and history from zero
    NA_TRY(cudaMemsetAsync(sc, 0, sizeof(double) * (S_COUNT + (size_t)iters + 1), st));
    if (x0 && x0 != x) NA_TRY(cudaMemcpyAsync(x, x0, sizeof(R) * n, cudaMemcpyDeviceToDevice, st));
    if (!x0) NA_TRY(cudaMemsetAsync(x, 0, sizeof(R) * n, st));
    {
        int l = 0;
        NA_TRY(launch_forward(p, x, r, st, &l));
        launches += l;
    }
    launch_pdl(k_residual0<R>, dim3(vb), dim3(vt), 0, st, d, r, m);
    {
        int l = 0;
        NA_TRY(launch_transpose(p, r, s, st, &l));
        launches += l;
    }
    launch_pdl(k_reduce_step<R, 2>, dim3(vb), dim3(vt), 0, st, s, n, (const R *)r, m, (const R *)x, pv,
               (R)(alpha * alpha), part, sc, resid, 0, alpha * alpha, cgls_tol2(p->precision));
    launches += 2;
    for (k = 1; k <= iters; ++k) {
        int l = 0;
        NA_TRY(launch_forward(p, pv, q, st, &l));
        launches += l;
        launch_pdl(k_reduce_step<R, 0>, dim3(vb), dim3(vt), 0, st, q, m, (const R *)pv, n, (const R *)nullptr,
                   (R *)nullptr, (R)0, part, sc, resid, k, 0.0, 0.0);
        launch_pdl(k_update_xr<R>, dim3(vb), dim3(vt), 0, st, x, pv, n, r, q, m, sc);
        NA_TRY(launch_transpose(p, r, s, st, &l));
        launches += l;
        launch_pdl(k_reduce_step<R, 1>, dim3(vb), dim3(vt), 0, st, s, n, (const R *)r, m, (const R *)x,
                   (R *)nullptr, (R)(alpha * alpha), part, sc, resid, k, 0.0, 0.0);
        launch_pdl(k_update_p<R>, dim3(vb), dim3(vt), 0, st, pv, s, n, sc);
        launches += 4;
        NA_TRY(cudaGetLastError());
    }
    NA_TRY(cudaGetLastError());
    if (resid_host) {
        NA_TRY(cudaMemcpyAsync(resid_host, resid, sizeof(double) * (iters + 1), cudaMemcpyDeviceToHost, st));
        NA_TRY(cudaStreamSynchronize(st));
    }
out:
#undef NA_TRY
    *nl = launches;
    return e;
}

cudaError_t run_cgls_noalloc(gm_plan *p, const void *d, const void *x0, void *x, double alpha, int iters,
                             double *resid_host, cudaStream_t s, int *nl) {
    if (p->precision != GM_F32)  // FP64 vectors (GM_F64, GM_DF64)
        return cgls_noalloc_t<double>(p, static_cast<const double *>(d), static_cast<const double *>(x0),
                                      static_cast<double *>(x), alpha, iters, resid_host, s, nl);
    return cgls_noalloc_t<float>(p, static_cast<const float *>(d), static_cast<const float *>(x0),
                                 static_cast<float *>(x), alpha, iters, resid_host, s, nl);
}

cudaError_t run_cgls(gm_plan *p, const void *d, const void *x0, void *x, double alpha, int iters, double *resid_host,
                     cudaStream_t s, int *nl) {
    if (p->precision != GM_F32)  // FP64 vectors (GM_F64, GM_DF64)
        return cgls_t<double>(p, static_cast<const double *>(d), static_cast<const double *>(x0),
                              static_cast<double *>(x), alpha, iters, resid_host, s, nl);
    return cgls_t<float>(p, static_cast<const float *>(d), static_cast<const float *>(x0), static_cast<float *>(x),
                         alpha, iters, resid_host, s, nl);
}

}  // namespace gm
