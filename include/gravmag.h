/*
 * gravmag.h -- C ABI of the GB300 fast BTTB gravity / magnetic operator.
 *
 * The library computes the forward product d = G m and the transpose product
 * m' = G^T d of the sensitivity matrix G of Hogue, Renaut & Vatankhah, "Fast
 * BTTB forward and transpose operators for 3-D gravity and magnetic data"
 * (arXiv 1912.06976):
 *
 *   Sec. 2 (Eqs. stationsij, prismspqr, Gslice, htilde) -- the geometry: sx * sy
 *     stations at the centres of the top faces of the unpadded cells, a volume
 *     of nx * ny * nz prisms with nx = sx + pxl + pxr, ny = sy + pyl + pyr
 *     (padding of Sec. 2.1.2, Eq. PaddedDistances), z positive down;
 *   Sec. 4 -- the entries: the gravity prism formula (Sec. 4.1) and the
 *     induced-magnetisation total-field formula (Sec. 4.2, Eq. magnetickernel);
 *   Sec. 3 (Eqs. GrviaT, Tcircpadded, Tcircpaddedgeneral, Wpadded, WTpadded,
 *     Ttran0, Ttran) and Algorithm multbttb -- the products through the
 *     block-circulant embedding and 2-D FFTs.
 *
 * Layouts (Eq. htilde, x fastest):
 *   model  m[r][q][p]  r < nz, q < ny, p < nx   (n = nx*ny*nz elements)
 *   data   d[j][i]     j < sy, i < sx           (m = sx*sy elements)
 * Element type: float for a GM_F32 handle, double for a GM_F64 or GM_DF64
 * handle.
 *
 * Units: gravity m in g/cm^3 and d in mGal (gamma = 6.67430e-3 mGal per
 * g/cm^3 per metre); magnetic m = susceptibility (SI) and d = total-field
 * anomaly in nT for a field of F nT (x North, y East, z down; inclination I
 * and declination D in degrees, induced magnetisation only).
 *
 * Ownership: the handle owns the spectra, the FFT twiddle tables and its
 * workspace, all allocated by the setup call on the device that is current
 * then; the caller owns every m / d buffer it passes.  Applies allocate
 * nothing, do not synchronise (except apply_forward_host /
 * apply_transpose_host) and are ordered on the CUDA stream passed in (NULL =
 * the legacy default stream).  The forward and the transpose products of a
 * handle have separate workspaces and host-call staging buffers: one forward
 * and one transpose (apply_forward / apply_transpose, or any of their
 * host-buffer variants, e.g. from two host threads) may run at the same time
 * on two streams (independent products, e.g. G m and G^T d of one step).
 * Other calls on one handle must not overlap in time: two forwards, two
 * transposes, gm_cgls / gm_cgls_noalloc (which use both products), and any
 * call while per-kernel timing is enabled; serialise them on one stream.
 * Distinct handles are independent.
 *
 * Errors: every call returns a gm_status (setup returns NULL and sets the
 * thread's last status).  No call faults the process on bad arguments.
 */
#ifndef GRAVMAG_H
#define GRAVMAG_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GM_API __attribute__((visibility("default")))
#else
#define GM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gm_plan *gm_handle;

typedef enum {
    GM_OK = 0,
    GM_EINVAL = 1,   /* bad argument: sizes, spacings, pointers, angles, aliasing */
    GM_ENOMEM = 2,   /* the plan does not fit in free device memory (or the set limit) */
    GM_ECUDA = 3,    /* a CUDA runtime call failed; the handle stays valid */
    GM_ETIMEOUT = 4, /* a bounded device-side wait gave up */
    GM_EDEVICE = 5,  /* a device-side check set the handle's error word */
    GM_ENODEV = 6    /* no usable CUDA device */
} gm_status;

typedef enum { GM_GRAVITY = 0, GM_MAGNETIC = 1 } gm_kind;
/* Apply precision.  GM_F32: FP32 vectors and arithmetic.  GM_F64: FP64
 * vectors and arithmetic.  GM_DF64: FP64 vectors, arithmetic on pairs of
 * FP32 values (h + l, a 48-bit significand, FP32's exponent range: values
 * between about 1e-30 and 1e38 in magnitude keep full accuracy), for GPUs
 * whose FP32 rate far exceeds their FP64 rate; its products agree with the
 * FP64 ones to about 1e-14 relative.  GM_DF64 runs only on the
 * register-codelet FFT lengths: it needs s + n - 1 <= 1024 in x and <= 768
 * in y (the plan always takes the smallest such length); larger grids
 * return GM_EINVAL at setup. */
typedef enum { GM_F32 = 0, GM_F64 = 1, GM_DF64 = 2 } gm_precision;

/* Full parameter record for grav_mag_setup_ex.  Sec. 2.1.2 and the parameter
 * table of App. A: stations, layers, cell sizes, left/right padding in x and y,
 * depth coordinates (z_blocks), and D, I, F for the magnetic kernel. */
typedef struct {
    int sx, sy, nz;         /* stations in x and y (>= 1); depth layers (>= 1)          */
    int pxl, pxr, pyl, pyr; /* padding cells before / after the stations (>= 0)          */
    double dx, dy;          /* cell sizes in x and y, metres (> 0)                        */
    double dz;              /* uniform layer thickness, used when zplanes == NULL (> 0)   */
    const double *zplanes;  /* optional HOST array of nz + 1 strictly increasing depths
                               (m) of the layer boundaries, zplanes[0] >= 0 (the stations
                               are at depth 0; Table of App. A, z_blocks); copied during
                               the call                                                   */
    int kind;               /* gm_kind                                                    */
    double incl_deg;        /* inclination I, |I| <= 90 (magnetic only)                   */
    double decl_deg;        /* declination D (magnetic only)                              */
    double F_nT;            /* field intensity F in nT (> 0; magnetic only)               */
    int precision;          /* gm_precision of the apply path; the setup is always FP64  */
} gm_params;

/* Set-up (Algorithms symBTTBFFT / BTTBFFT of App. B): evaluates the prism
 * entries of every depth layer in FP64 on the device, builds the circulant
 * generators of Eqs. Tcircpadded / Tcircpaddedgeneral and stores their 2-D
 * FFTs.  nx, ny are the STATION counts s_x, s_y (= unpadded cells); px, py
 * pad cells on EACH side; dz the uniform layer thickness; kind a gm_kind;
 * incl_deg, decl_deg are ignored for gravity.  F = 50000 nT, FP32 applies.
 * Set-up blocks the calling thread and synchronises the current device: when
 * it returns, every table and spectrum is on the device, so the handle can be
 * used on any stream.  Returns NULL on error (see gm_last_status /
 * gm_last_error). */
GM_API gm_handle grav_mag_setup(int nx, int ny, int nz, double dx, double dy, double dz, int px, int py,
                         int kind, double incl_deg, double decl_deg);

/* Set-up with the full parameter record (asymmetric padding, variable layer
 * depths, F, apply precision).  NULL on error. */
GM_API gm_handle grav_mag_setup_ex(const gm_params *p);

/* Forward product d = G m (Algorithm multbttb, t = 1; Eq. GrviaT with W of
 * Eq. Wpadded): m_dev is a device array of n elements, d_dev one of m
 * elements, in the handle's precision; d is overwritten.  m_dev and d_dev
 * must not overlap (GM_EINVAL).  stream: a cudaStream_t or NULL. */
GM_API gm_status apply_forward(gm_handle h, const void *m_dev, void *d_dev, void *stream);

/* Transpose product m' = G^T d (Algorithm multbttb, t = 2; Eqs. Ttran0, Ttran
 * and WTpadded; realised with the complex conjugate of the forward spectra,
 * which equals the FFT of the index-reversed generator because the
 * generator is real).  d_dev: m elements, m_dev: n elements, overwritten. */
GM_API gm_status apply_transpose(gm_handle h, const void *d_dev, void *m_dev, void *stream);

/* The same products from and to HOST buffers (m_host: n elements, d_host: m
 * elements, in the handle's precision; the two must not overlap, GM_EINVAL).
 * Each direction has two model-sized device staging buffers used in turn, a
 * data-sized one, and two internal streams: the model goes over the host link
 * by the copy engine on one of them while the product runs on the other, so a
 * call's model copy overlaps the kernels of the calls next to it.  `stream`
 * waits for the call's last copy: the output is complete once `stream` has
 * reached the end of the call.  These two calls also synchronise `stream`
 * before returning.  Page-locked buffers (cudaHostAlloc / cudaHostRegister,
 * e.g. torch pin_memory) give the full host-link rate; pageable memory works
 * too.  With GM_HOST_DIRECT=1 in the environment and both buffers
 * page-locked, the kernels instead read the input and write the output in
 * place through the GPU's view of host memory, on `stream`. */
GM_API gm_status apply_forward_host(gm_handle h, const void *m_host, void *d_host, void *stream);
GM_API gm_status apply_transpose_host(gm_handle h, const void *d_host, void *m_host, void *stream);

/* The same calls without the final synchronisation: they enqueue the work and
 * return.  The output is complete once `stream` has reached the end of the
 * call (cudaStreamSynchronize, an event); until then both host buffers must
 * stay allocated and the input unchanged.  Unlike apply_forward, the call may
 * read the input and write the output before `stream` reaches it (the
 * internal streams run ahead while consecutive calls of one direction come on
 * one stream), so earlier work on `stream` must not write the input or use
 * the output buffer.  Inside a stream capture the copies and the product are
 * captured on `stream` in order.  With page-locked buffers the call returns at
 * once; with pageable buffers the copies block the calling thread as
 * cudaMemcpyAsync does.  Calls of one direction must be ordered (one stream,
 * or events), like apply_forward / apply_transpose. */
GM_API gm_status apply_forward_host_async(gm_handle h, const void *m_host, void *d_host, void *stream);
GM_API gm_status apply_transpose_host_async(gm_handle h, const void *d_host, void *m_host, void *stream);

/* Releases everything the handle owns (synchronises its device first).
 * NULL is accepted and returns GM_OK. */
GM_API gm_status grav_mag_destroy(gm_handle h);

/* Sizes and memory of a plan. */
typedef struct {
    int sx, sy, nz, nx, ny;  /* stations, layers and padded cells                        */
    int fft_nx, fft_ny;      /* FFT lengths N'_x >= sx + nx - 1, N'_y >= sy + ny - 1      */
    int spec_nx;             /* N'_x / 2 + 1 columns kept of each real-input transform   */
    int kind, precision;
    int64_t n_model, n_data; /* n and m                                                   */
    size_t spectrum_bytes;   /* resident spectra                                          */
    size_t workspace_bytes;  /* resident workspace (intermediates + host-call staging)    */
    double setup_ms;         /* device time of the set-up kernels                         */
    int spectrum_real;       /* 1: stored spectra are the real even spectra of the
                                station-centred generator (gravity, equal padding on both
                                sides), a quarter of the complex bytes; 0: complex        */
} gm_info;

GM_API gm_status gm_get_info(gm_handle h, gm_info *out);

/* Copies the spectra to host memory: out holds spec_nx * nz * fft_ny complex
 * values (interleaved re, im) in the handle's vector type (float for GM_F32,
 * double for GM_F64; GM_DF64 spectra are returned as doubles h + l), ordered [kx][r][ky],
 * i.e. the 2-D FFT of layer r's circulant generator at frequency (kx, ky).
 * bytes must be at least that size (2 * element size * spec_nx * nz * fft_ny).
 * A handle that stores real even spectra (gm_info.spectrum_real) expands them
 * on the host into this same complex form. */
GM_API gm_status gm_copy_spectrum(gm_handle h, void *host_out, size_t bytes);

/* Smallest even integer >= max(n, 2) whose prime factors are all in
 * {2, 3, 5, 7}: the FFT length the plan uses per axis for a linear
 * convolution of support n (any length >= n is exact, Sec. 3).  Host only.
 * Returns -1 for n < 1 or n > 2^24. */
GM_API int gm_fft_length(int n);

/* Checks a parameter record without touching the device (GM_OK / GM_EINVAL). */
GM_API gm_status gm_validate_params(const gm_params *p);

/* Caps the device bytes a set-up may allocate (0 = no cap beyond free
 * memory); a plan above the cap fails with GM_ENOMEM before allocating. */
GM_API void gm_set_memory_limit(size_t bytes);

/* Tikhonov-regularised least squares (min ||G x - d||^2 + alpha^2 ||x||^2)
 * by CGLS: each iteration applies G once and G^T once; the vector updates,
 * dot products (accumulated in FP64) and step lengths stay on the device, so
 * the loop never waits for the host.  d_dev: m elements; x0_dev: n elements
 * or NULL for a zero start; x_dev: n elements, receives the iterate after
 * `iters` iterations (may equal x0_dev).  resid_host, if not NULL, receives
 * iters + 1 values of ||G x_k - d||_2 (k = 0..iters; synchronises the stream
 * at the end).  Scratch: six vectors held by the handle, allocated on the
 * first call (so the first call is not capturable in a CUDA graph). */
GM_API gm_status gm_cgls(gm_handle h, const void *d_dev, const void *x0_dev, void *x_dev, double alpha,
                  int iters, double *resid_host, void *stream);

/* CGLS exactly like gm_cgls, but without allocating any device memory.  This
 * entry point has no counterpart in the paper; it exists for callers that
 * cannot call cudaMalloc when they solve: processes whose GPU memory is
 * entirely reserved by a framework's pooling allocator, latency-critical loops
 * that cannot afford the device-wide synchronisation cudaMalloc and cudaFree
 * may cause, and long-running services that must not grow their device
 * footprint after start-up.  Its scratch is a fixed 16 MiB array compiled into
 * the library (gm_cgls_noalloc_capacity() bytes), which every GPU that loads
 * the library holds until the process exits.  A grid needs
 * (2 n + 2 m) * element size + 8 * (1032 + iters + 1) bytes, rounded up to 256
 * for the vectors; larger requests fail with GM_EINVAL and a message, before
 * anything runs.  The first call on a device looks up the array's device
 * address (a one-time set-up per device, done with that device current); make
 * that first call before any stream capture.  All calls in the process share
 * the array and it keeps the last call's contents (each call clears what it
 * needs cleared), so calls that overlap on the GPU race: serialise them.
 * Arguments and results are those of gm_cgls. */
GM_API gm_status gm_cgls_noalloc(gm_handle h, const void *d_dev, const void *x0_dev, void *x_dev, double alpha,
                                 int iters, double *resid_host, void *stream);
GM_API size_t gm_cgls_noalloc_capacity(void);

/* Thread-local status and message of the last failing call of this thread. */
GM_API gm_status gm_last_status(void);
GM_API const char *gm_last_error(void);
GM_API const char *gm_status_string(gm_status s);

/* Number of kernels the last apply / CGLS call on this handle launched. */
GM_API int gm_last_launch_count(gm_handle h);

/* Per-kernel device timing of the handle's own launches (tracing).  While
 * enabled with a capacity > 0, every kernel the handle launches is bracketed by
 * two CUDA events recorded on the launching stream (up to `capacity` launches;
 * later launches run untimed).  gm_kernel_times synchronises those events and
 * returns, per kernel, its launch count and summed device time since the last
 * query (then resets).  capacity = 0 disables timing and frees the events. */
typedef struct {
    char name[32];  /* kernel name, e.g. "fwd_cols_mac" */
    int launches;
    double total_ms;
} gm_kernel_time;

GM_API gm_status gm_enable_timing(gm_handle h, int capacity);
GM_API int gm_kernel_times(gm_handle h, gm_kernel_time *out, int max_entries);

#ifdef __cplusplus
}
#endif

#endif /* GRAVMAG_H */
