// capi.cu -- the extern "C" boundary declared in include/gravmag.h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "gm_fast_ops.h"
#include "gm_plan.h"

namespace {

thread_local gm_status g_last_status = GM_OK;
thread_local char g_last_msg[512] = "";
size_t g_mem_limit = 0;

gm_status fail(gm_status s, const char *fmt, ...) {
    g_last_status = s;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_msg, sizeof(g_last_msg), fmt, ap);
    va_end(ap);
    return s;
}

gm_status ok() {
    g_last_status = GM_OK;
    g_last_msg[0] = 0;
    return GM_OK;
}

gm_status cuda_fail(cudaError_t e, const char *where) {
    cudaGetLastError();  // clear a sticky-free error so the handle stays usable
    return fail(GM_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

bool is_smooth7(int n) {
    for (int p : {2, 3, 5, 7})
        while (n % p == 0) n /= p;
    return n == 1;
}

// Scoped switch to the handle's device.
struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            changed = cudaSetDevice(dev) == cudaSuccess;
        }
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr double kGamma = 6.67430e-3;  // mGal per (g/cm^3 m)
constexpr int kMaxFft = 4800;          // one FFT column / row must fit a CTA's shared memory in FP64

// GM_GENERIC_FFT=1 in the environment selects the generic kernels for every length.
bool fast_disabled() {
    const char *v = std::getenv("GM_GENERIC_FFT");
    return v && v[0] == '1';
}

}  // namespace

namespace gm {

const char *const kKernelNames[K_COUNT] = {"fwd_rows_r2c", "fwd_cols_mac", "fwd_rows_c2r", "tr_rows_r2c",
                                           "tr_cols",      "tr_rows_c2r",  "cgls_vec",     "fwd_cols_inv"};

bool make_radices(int N, FftDesc &d) {
    d.N = N;
    d.npass = 0;
    int n = N;
    const int order[] = {8, 4, 2, 3, 5, 7};
    for (int r : order) {
        while (n % r == 0) {
            if (d.npass >= kMaxPasses) return false;
            d.radix[d.npass++] = r;
            n /= r;
        }
    }
    return n == 1;
}

cudaError_t make_twiddles(int N, int precision, void **dev_out) {
    *dev_out = nullptr;
    const bool f64 = precision == GM_F64, df = precision == GM_DF64;
    size_t elt = (f64 || df) ? sizeof(double2) : sizeof(float2);
    std::string host(elt * (size_t)N, '\0');
    for (int e = 0; e < N; ++e) {
        // exp(-2 pi i e / N) in long double, rounded once
        long double ang = -2.0L * 3.14159265358979323846264338327950288L * (long double)e / (long double)N;
        long double c = cosl(ang), s = sinl(ang);
        if (f64) {
            double2 v = make_double2((double)c, (double)s);
            std::memcpy(&host[elt * e], &v, elt);
        } else if (df) {  // each part rounded to the nearest FP32 pair h + l; order {re.h, im.h, re.l, im.l}
            const float ch = (float)c, sh = (float)s;
            const float v[4] = {ch, sh, (float)(c - (long double)ch), (float)(s - (long double)sh)};
            std::memcpy(&host[elt * e], v, elt);
        } else {
            float2 v = make_float2((float)c, (float)s);
            std::memcpy(&host[elt * e], &v, elt);
        }
    }
    cudaError_t err = cudaMalloc(dev_out, elt * (size_t)N);
    if (err != cudaSuccess) return err;
    err = cudaMemcpy(*dev_out, host.data(), elt * (size_t)N, cudaMemcpyHostToDevice);
    // A copy from pageable host memory may return before the data reaches the device, and it
    // is ordered only on the legacy default stream: the set-up kernels run on a non-blocking
    // stream and callers may apply on any stream, so wait for the table to land.
    if (err == cudaSuccess) err = cudaDeviceSynchronize();
    return err;
}

}  // namespace gm

static void free_timing(gm_plan *p) {
    for (cudaEvent_t e : p->tev) cudaEventDestroy(e);
    p->tev.clear();
    p->tkid.clear();
    p->tused = 0;
}

static void free_plan(gm_plan *p) {
    if (!p) return;
    free_timing(p);
    cudaFree(p->spec);
    cudaFree(p->work_big);
    cudaFree(p->work_small);
    cudaFree(p->work_big_tr);
    cudaFree(p->work_small_tr);
    cudaFree(p->work_part);
    cudaFree(p->work_counters);
    for (gm_plan::HostPipe *hp : {&p->host_fwd, &p->host_tr}) {
        cudaFree(hp->stage[0]);
        cudaFree(hp->stage[1]);
        cudaFree(hp->stage_small);
        if (hp->ks) cudaStreamDestroy(hp->ks);
        if (hp->cs) cudaStreamDestroy(hp->cs);
        for (cudaEvent_t e : {hp->fork, hp->done, hp->ready[0], hp->ready[1], hp->freed[0], hp->freed[1]})
            if (e) cudaEventDestroy(e);
    }
    cudaFree(p->tw_x);
    cudaFree(p->tw_y);
    cudaFree(p->cgls_buf);
    delete p;
}

template <typename R>
void expand_real_spectrum(const gm_plan *h, const R *E, R *out) {
    // T[kx][r][ky] = w(kx, ky) E[kx][r][min(ky, N'y - ky)], w = exp(+2 pi i (pxl kx / N'x + pyl ky / N'y))
    const gm::Geo &g = h->geo;
    const int H = g.NPy / 2 + 1;
    for (int kx = 0; kx < g.Kx; ++kx)
        for (int ky = 0; ky < g.NPy; ++ky) {
            const double ph = 2.0 * kPi *
                              ((double)(((long long)g.pxl * kx) % g.NPx) / g.NPx +
                               (double)(((long long)g.pyl * ky) % g.NPy) / g.NPy);
            const double wr = std::cos(ph), wi = std::sin(ph);
            for (int r = 0; r < g.nz; ++r) {
                const double e = (double)E[((size_t)kx * g.nz + r) * H + (ky <= g.NPy / 2 ? ky : g.NPy - ky)];
                R *o = out + 2 * (((size_t)kx * g.nz + r) * g.NPy + ky);
                o[0] = (R)(wr * e);
                o[1] = (R)(wi * e);
            }
        }
}

extern "C" {

int gm_fft_length(int n) {
    if (n < 1 || n > (1 << 24)) return -1;
    int m = n < 2 ? 2 : n;
    if (m & 1) ++m;
    while (!is_smooth7(m)) m += 2;
    return m;
}

gm_status gm_validate_params(const gm_params *p) {
    if (!p) return fail(GM_EINVAL, "params is NULL");
    if (p->sx < 1 || p->sy < 1 || p->nz < 1) return fail(GM_EINVAL, "sx, sy, nz must be >= 1");
    if (p->nz > 65535) return fail(GM_EINVAL, "nz must be <= 65535");
    if (p->pxl < 0 || p->pxr < 0 || p->pyl < 0 || p->pyr < 0) return fail(GM_EINVAL, "padding must be >= 0");
    if (!(p->dx > 0) || !(p->dy > 0) || !std::isfinite(p->dx) || !std::isfinite(p->dy))
        return fail(GM_EINVAL, "dx, dy must be finite and > 0");
    if (p->kind != GM_GRAVITY && p->kind != GM_MAGNETIC) return fail(GM_EINVAL, "kind must be GM_GRAVITY or GM_MAGNETIC");
    if (p->precision != GM_F32 && p->precision != GM_F64 && p->precision != GM_DF64)
        return fail(GM_EINVAL, "precision must be GM_F32, GM_F64 or GM_DF64");
    if (p->zplanes) {
        if (!(p->zplanes[0] >= 0) || !std::isfinite(p->zplanes[0])) return fail(GM_EINVAL, "zplanes[0] must be >= 0");
        for (int k = 0; k < p->nz; ++k)
            if (!(p->zplanes[k + 1] > p->zplanes[k]) || !std::isfinite(p->zplanes[k + 1]))
                return fail(GM_EINVAL, "zplanes must be finite and strictly increasing");
    } else if (!(p->dz > 0) || !std::isfinite(p->dz)) {
        return fail(GM_EINVAL, "dz must be finite and > 0");
    }
    if (p->kind == GM_MAGNETIC) {
        if (!(std::fabs(p->incl_deg) <= 90.0)) return fail(GM_EINVAL, "|inclination| must be <= 90 degrees");
        if (!std::isfinite(p->decl_deg)) return fail(GM_EINVAL, "declination must be finite");
        if (!(p->F_nT > 0) || !std::isfinite(p->F_nT)) return fail(GM_EINVAL, "F must be finite and > 0");
    }
    const long long nx = (long long)p->sx + p->pxl + p->pxr, ny = (long long)p->sy + p->pyl + p->pyr;
    const long long Nx = p->sx + nx - 1, Ny = p->sy + ny - 1;
    if (Nx > kMaxFft || Ny > kMaxFft) return fail(GM_EINVAL, "s + n - 1 per axis must be <= %d", kMaxFft);
    const int Px = gm_fft_length((int)Nx), Py = gm_fft_length((int)Ny);
    if (Px < 0 || Py < 0 || Px > kMaxFft || Py > kMaxFft)
        return fail(GM_EINVAL, "FFT length above %d", kMaxFft);
    if (nx * ny * (long long)p->nz > (1LL << 40)) return fail(GM_EINVAL, "volume too large");
    return ok();
}

void gm_set_memory_limit(size_t bytes) { g_mem_limit = bytes; }

// NVTX range around one C-ABI call (the kernels it launches carry ranges of their own).
struct NvtxScope {
    explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope &) = delete;
    NvtxScope &operator=(const NvtxScope &) = delete;
};

gm_handle grav_mag_setup_ex(const gm_params *prm) {
    NvtxScope nv("grav_mag_setup_ex");
    if (gm_validate_params(prm) != GM_OK) return nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        fail(GM_ENODEV, "no CUDA device");
        return nullptr;
    }
    gm_plan *p = new (std::nothrow) gm_plan();
    if (!p) {
        fail(GM_ENOMEM, "host allocation failed");
        return nullptr;
    }
    cudaGetDevice(&p->device);
    p->kind = prm->kind;
    p->precision = prm->precision;
    gm::Geo &g = p->geo;
    g.sx = prm->sx; g.sy = prm->sy; g.nz = prm->nz;
    g.pxl = prm->pxl; g.pyl = prm->pyl;
    p->pxr = prm->pxr; p->pyr = prm->pyr;
    g.nx = prm->sx + prm->pxl + prm->pxr;
    g.ny = prm->sy + prm->pyl + prm->pyr;
    g.nyp = (g.ny + 15) / 16 * 16;  // intermediate column pitch: whole 128-byte lines per column
    p->Nx = g.sx + g.nx - 1;
    p->Ny = g.sy + g.ny - 1;
    // FFT lengths: the smallest lengths >= Nx, Ny that the register-codelet kernels are built for
    // when both are within 25% of the smallest even 7-smooth lengths (always, for GM_DF64, which
    // has no other kernels); otherwise those 7-smooth lengths (generic kernels).  Any length >= N
    // gives the same products (Sec. 3).
    {
        const int sx7 = gm_fft_length(p->Nx), sy7 = gm_fft_length(p->Ny);
        const int lx = fast_disabled() ? 0 : gm::fast_ladder_length(p->Nx, false);
        const int ly = fast_disabled() ? 0 : gm::fast_ladder_length(p->Ny, true);
        const bool ladder =
            lx && ly && (prm->precision == GM_DF64 || (4 * lx <= 5 * sx7 && 4 * ly <= 5 * sy7));
        g.NPx = ladder ? lx : sx7;
        g.NPy = ladder ? ly : sy7;
    }
    g.Kx = g.NPx / 2 + 1;
    p->dx = prm->dx; p->dy = prm->dy;
    p->zplanes.resize(g.nz + 1);
    for (int k = 0; k <= g.nz; ++k) p->zplanes[k] = prm->zplanes ? prm->zplanes[k] : k * prm->dz;
    p->incl_deg = prm->incl_deg; p->decl_deg = prm->decl_deg; p->F_nT = prm->F_nT;
    if (p->kind == GM_GRAVITY) {
        p->coef[0] = kGamma;
    } else {
        // Eq. magnetickernel with Fhat = (cos I cos D, cos I sin D, sin I), x North, y East, z down:
        // (F/4pi) [2 m n Lx + 2 l n Ly + 2 l m Lz + (n^2 - l^2) Ax + (n^2 - m^2) Ay]
        const double I = p->incl_deg * kPi / 180.0, D = p->decl_deg * kPi / 180.0;
        const double l = std::cos(I) * std::cos(D), m = std::cos(I) * std::sin(D), n = std::sin(I);
        const double H = p->F_nT / (4.0 * kPi);
        p->coef[0] = H * 2.0 * m * n;
        p->coef[1] = H * 2.0 * l * n;
        p->coef[2] = H * 2.0 * l * m;
        p->coef[3] = H * (n * n - l * l);
        p->coef[4] = H * (n * n - m * m);
    }
    if (!gm::make_radices(g.NPx, p->fx) || !gm::make_radices(g.NPy, p->fy)) {
        free_plan(p);
        fail(GM_EINVAL, "internal: FFT length not 7-smooth");
        return nullptr;
    }
    // Memory guard (the paper's memory-safety test, Sec. 6): resident + set-up peak.
    const size_t cel = prm->precision == GM_F32 ? sizeof(float2) : sizeof(double2);
    const size_t rel = prm->precision == GM_F32 ? sizeof(float) : sizeof(double);
    const size_t nspec = (size_t)g.Kx * g.nz * g.NPy;
    p->spec_bytes = cel * nspec;
    const size_t big = cel * (size_t)g.Kx * g.nz * g.nyp;
    const size_t small = cel * (size_t)g.Kx * g.sy;
    const size_t n_model = (size_t)g.nx * g.ny * g.nz, n_data = (size_t)g.sx * g.sy;
    p->fast = !fast_disabled() && gm::fast_path_supported(g.NPx, g.NPy);
    if (prm->precision == GM_DF64 && !p->fast) {
        free_plan(p);
        fail(GM_EINVAL, "GM_DF64 needs FFT lengths on the register-codelet ladder (here %d x %d)", g.NPx, g.NPy);
        return nullptr;
    }
    // gravity with the same padding on both sides: real even spectra, a quarter of the bytes
    // (register-codelet path; GM_COMPLEX_SPECTRA=1 keeps the complex form)
    {
        const char *cs = std::getenv("GM_COMPLEX_SPECTRA");
        p->spec_real = p->fast && p->kind == GM_GRAVITY && g.pxl == p->pxr && g.pyl == p->pyr &&
                       !(cs && cs[0] && cs[0] != '0');
    }
    if (p->spec_real) p->spec_bytes = rel * (size_t)g.Kx * g.nz * (g.NPy / 2 + 1);
    size_t part = 0, ncount = 0;
    if (p->fast) {
        gm::fast_plan_groups(p);
        part = cel * (size_t)p->fast_groups_fwd * g.Kx * g.NPy;
        ncount = (size_t)gm::fast_column_groups(p);
    }
    p->work_bytes = 2 * (big + small) + part + 2 * rel * (2 * n_model + n_data);
    const size_t setup_peak = sizeof(double) * ((size_t)(p->Nx + 1) * (p->Ny + 1) * g.nz +
                                                (size_t)g.NPx * g.NPy * g.nz) +
                              sizeof(double2) * nspec + 4 * sizeof(double2) * (g.NPx + g.NPy);
    const size_t need = p->spec_bytes + p->work_bytes + setup_peak;
    size_t freeb = 0, totalb = 0;
    cudaError_t e = cudaMemGetInfo(&freeb, &totalb);
    if (e != cudaSuccess) {
        free_plan(p);
        cuda_fail(e, "cudaMemGetInfo");
        return nullptr;
    }
    if (need > freeb || (g_mem_limit && need > g_mem_limit)) {
        free_plan(p);
        fail(GM_ENOMEM, "plan needs %zu bytes, %zu free%s", need, freeb, g_mem_limit ? " (or above the set limit)" : "");
        return nullptr;
    }
#define SETUP_TRY(x, what)                 \
    do {                                   \
        cudaError_t e_ = (x);              \
        if (e_ != cudaSuccess) {           \
            free_plan(p);                  \
            cuda_fail(e_, what);           \
            return nullptr;                \
        }                                  \
    } while (0)
    SETUP_TRY(gm::make_twiddles(g.NPx, prm->precision, &p->tw_x), "twiddles x");
    SETUP_TRY(gm::make_twiddles(g.NPy, prm->precision, &p->tw_y), "twiddles y");
    p->fx.tw = p->tw_x;
    p->fy.tw = p->tw_y;
    SETUP_TRY(cudaMalloc(&p->spec, p->spec_bytes), "spectra");
    SETUP_TRY(cudaMalloc(&p->work_big, big), "workspace");
    SETUP_TRY(cudaMalloc(&p->work_small, small), "workspace");
    SETUP_TRY(cudaMalloc(&p->work_big_tr, big), "workspace");
    SETUP_TRY(cudaMalloc(&p->work_small_tr, small), "workspace");
    if (part) SETUP_TRY(cudaMalloc(&p->work_part, part), "workspace");
    if (ncount) {
        SETUP_TRY(cudaMalloc(&p->work_counters, sizeof(unsigned int) * ncount), "workspace");
        SETUP_TRY(cudaMemset(p->work_counters, 0, sizeof(unsigned int) * ncount), "workspace");
        // the memset is ordered on the legacy default stream only; applies may come on any stream
        SETUP_TRY(cudaDeviceSynchronize(), "workspace");
    }
    for (gm_plan::HostPipe *hp : {&p->host_fwd, &p->host_tr}) {
        SETUP_TRY(cudaMalloc(&hp->stage[0], rel * n_model), "staging");
        SETUP_TRY(cudaMalloc(&hp->stage[1], rel * n_model), "staging");
        SETUP_TRY(cudaMalloc(&hp->stage_small, rel * n_data), "staging");
        SETUP_TRY(cudaStreamCreateWithFlags(&hp->ks, cudaStreamNonBlocking), "stream");
        SETUP_TRY(cudaStreamCreateWithFlags(&hp->cs, cudaStreamNonBlocking), "stream");
        for (cudaEvent_t *e : {&hp->fork, &hp->done, &hp->ready[0], &hp->ready[1], &hp->freed[0], &hp->freed[1]})
            SETUP_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming), "event");
    }
    cudaStream_t s;
    SETUP_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream");
    cudaError_t be = gm::build_spectra(p, s);
    cudaStreamDestroy(s);
    if (be != cudaSuccess) {
        free_plan(p);
        cuda_fail(be, "set-up kernels");
        return nullptr;
    }
#undef SETUP_TRY
    ok();
    return p;
}

gm_handle grav_mag_setup(int nx, int ny, int nz, double dx, double dy, double dz, int px, int py, int kind,
                         double incl_deg, double decl_deg) {
    gm_params prm;
    std::memset(&prm, 0, sizeof(prm));
    prm.sx = nx; prm.sy = ny; prm.nz = nz;
    prm.pxl = prm.pxr = px;
    prm.pyl = prm.pyr = py;
    prm.dx = dx; prm.dy = dy; prm.dz = dz;
    prm.zplanes = nullptr;
    prm.kind = kind;
    prm.incl_deg = kind == GM_MAGNETIC ? incl_deg : 90.0;
    prm.decl_deg = kind == GM_MAGNETIC ? decl_deg : 0.0;
    prm.F_nT = 50000.0;
    prm.precision = GM_F32;
    return grav_mag_setup_ex(&prm);
}

static bool overlaps(const void *a, size_t na, const void *b, size_t nb) {
    const char *pa = static_cast<const char *>(a), *pb = static_cast<const char *>(b);
    return pa < pb + nb && pb < pa + na;
}

static gm_status check_apply(gm_handle h, const void *in, size_t nin, const void *out, size_t nout) {
    if (!h) return fail(GM_EINVAL, "handle is NULL");
    if (!in || !out) return fail(GM_EINVAL, "NULL buffer");
    const size_t rel = h->precision == GM_F32 ? sizeof(float) : sizeof(double);
    if (overlaps(in, nin * rel, out, nout * rel)) return fail(GM_EINVAL, "input and output overlap");
    return GM_OK;
}

gm_status apply_forward(gm_handle h, const void *m_dev, void *d_dev, void *stream) {
    NvtxScope nv("apply_forward");
    if (!h) return fail(GM_EINVAL, "handle is NULL");
    const size_t n = (size_t)h->geo.nx * h->geo.ny * h->geo.nz, m = (size_t)h->geo.sx * h->geo.sy;
    gm_status st = check_apply(h, m_dev, n, d_dev, m);
    if (st != GM_OK) return st;
    DeviceGuard dg(h->device);
    h->host_fwd.chained = false;  // the next host-buffer forward waits for this one's stream
    int nl = 0;
    cudaError_t e = gm::launch_forward(h, m_dev, d_dev, static_cast<cudaStream_t>(stream), &nl);
    h->last_launches = nl;
    if (e != cudaSuccess) return cuda_fail(e, "apply_forward");
    return ok();
}

gm_status apply_transpose(gm_handle h, const void *d_dev, void *m_dev, void *stream) {
    NvtxScope nv("apply_transpose");
    if (!h) return fail(GM_EINVAL, "handle is NULL");
    const size_t n = (size_t)h->geo.nx * h->geo.ny * h->geo.nz, m = (size_t)h->geo.sx * h->geo.sy;
    gm_status st = check_apply(h, d_dev, m, m_dev, n);
    if (st != GM_OK) return st;
    DeviceGuard dg(h->device);
    h->host_tr.chained = false;
    int nl = 0;
    cudaError_t e = gm::launch_transpose(h, d_dev, m_dev, static_cast<cudaStream_t>(stream), &nl);
    h->last_launches = nl;
    if (e != cudaSuccess) return cuda_fail(e, "apply_transpose");
    return ok();
}

// Device address of a page-locked host buffer the GPU can access directly, or nullptr.
static void *device_view_of_pinned(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// One host-buffer product.  Page-locked buffers with GM_HOST_DIRECT=1: the kernels use them in
// place on `stream`.  Inside a stream capture: copy in, product and copy out on `stream`, through
// the direction's first staging buffer.  Otherwise the direction's pipeline: the model copy runs on
// the copy stream (forward: in, into the staging buffer of this call; transpose: out, from it), the
// product on the kernel stream (which also reads or writes the data vector, in place when it is
// page-locked, else through the small staging buffer), and `stream` waits for the call's end.  The
// two staging buffers alternate, so the model copy of one call overlaps the kernels of the next.
// The internal streams wait for `stream` to reach the call unless the previous call of this
// direction came on the same stream with nothing of this direction in between (it already made
// `stream` wait for it, and the kernel stream keeps the calls in order).
static gm_status host_apply(gm_handle h, const void *in_host, void *out_host, void *stream, bool fwd, bool sync) {
    NvtxScope nv(fwd ? (sync ? "apply_forward_host" : "apply_forward_host_async")
                     : (sync ? "apply_transpose_host" : "apply_transpose_host_async"));
    if (!h) return fail(GM_EINVAL, "handle is NULL");
    if (!in_host || !out_host) return fail(GM_EINVAL, "NULL buffer");
    const size_t rel = h->precision == GM_F32 ? sizeof(float) : sizeof(double);
    const size_t n = (size_t)h->geo.nx * h->geo.ny * h->geo.nz, m = (size_t)h->geo.sx * h->geo.sy;
    const size_t nin = fwd ? n : m, nout = fwd ? m : n;
    if (overlaps(in_host, nin * rel, out_host, nout * rel)) return fail(GM_EINVAL, "input and output overlap");
    DeviceGuard dg(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    gm_plan::HostPipe &hp = fwd ? h->host_fwd : h->host_tr;
    int nl = 0;
    cudaError_t e = cudaSuccess;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return cuda_fail(e, "stream query");
    const char *direct = std::getenv("GM_HOST_DIRECT");
    void *in_dev = nullptr, *out_dev = nullptr;
    if (direct && direct[0] && direct[0] != '0') {
        in_dev = device_view_of_pinned(in_host);
        out_dev = device_view_of_pinned(out_host);
    }
    const bool chained = hp.chained && hp.chain == s;
    hp.chained = false;  // set again below once this call has been enqueued in full
#define HP_TRY(x, what)                                 \
    do {                                                \
        e = (x);                                        \
        if (e != cudaSuccess) return cuda_fail(e, what); \
    } while (0)
    if (in_dev && out_dev) {
        HP_TRY(fwd ? gm::launch_forward(h, in_dev, out_dev, s, &nl) : gm::launch_transpose(h, in_dev, out_dev, s, &nl),
               "apply");
    } else if (cap != cudaStreamCaptureStatusNone) {
        void *big = hp.stage[0], *small = hp.stage_small;
        HP_TRY(cudaMemcpyAsync(fwd ? big : small, in_host, rel * nin, cudaMemcpyHostToDevice, s), "host-to-device copy");
        HP_TRY(fwd ? gm::launch_forward(h, big, small, s, &nl) : gm::launch_transpose(h, small, big, s, &nl), "apply");
        HP_TRY(cudaMemcpyAsync(out_host, fwd ? small : big, rel * nout, cudaMemcpyDeviceToHost, s),
               "device-to-host copy");
    } else {
        const int b = hp.next;
        if (!chained) {
            HP_TRY(cudaEventRecord(hp.fork, s), "event record");
            HP_TRY(cudaStreamWaitEvent(hp.ks, hp.fork, 0), "stream wait");
        }
        // The data vector (m elements) is read or written in place by the kernels when its buffer
        // is page-locked: a copy-engine transfer of it would queue behind the other direction's
        // model copy on the same engine.
        if (fwd) {
            void *d_view = device_view_of_pinned(out_host);
            // copy stream: model in, once the call two back has finished with this staging buffer
            HP_TRY(cudaStreamWaitEvent(hp.cs, hp.freed[b], 0), "stream wait");
            HP_TRY(cudaMemcpyAsync(hp.stage[b], in_host, rel * n, cudaMemcpyHostToDevice, hp.cs), "host-to-device copy");
            HP_TRY(cudaEventRecord(hp.ready[b], hp.cs), "event record");
            // kernel stream: product, data out
            HP_TRY(cudaStreamWaitEvent(hp.ks, hp.ready[b], 0), "stream wait");
            HP_TRY(gm::launch_forward(h, hp.stage[b], d_view ? d_view : hp.stage_small, hp.ks, &nl), "apply");
            HP_TRY(cudaEventRecord(hp.freed[b], hp.ks), "event record");
            if (!d_view)
                HP_TRY(cudaMemcpyAsync(out_host, hp.stage_small, rel * m, cudaMemcpyDeviceToHost, hp.ks),
                       "device-to-host copy");
            HP_TRY(cudaEventRecord(hp.done, hp.ks), "event record");
        } else {
            const void *d_view = device_view_of_pinned(in_host);
            // kernel stream: data in, product into this call's staging buffer
            if (!d_view)
                HP_TRY(cudaMemcpyAsync(hp.stage_small, in_host, rel * m, cudaMemcpyHostToDevice, hp.ks),
                       "host-to-device copy");
            HP_TRY(cudaStreamWaitEvent(hp.ks, hp.freed[b], 0), "stream wait");
            HP_TRY(gm::launch_transpose(h, d_view ? d_view : hp.stage_small, hp.stage[b], hp.ks, &nl), "apply");
            HP_TRY(cudaEventRecord(hp.ready[b], hp.ks), "event record");
            // copy stream: model out
            HP_TRY(cudaStreamWaitEvent(hp.cs, hp.ready[b], 0), "stream wait");
            HP_TRY(cudaMemcpyAsync(out_host, hp.stage[b], rel * n, cudaMemcpyDeviceToHost, hp.cs),
                   "device-to-host copy");
            HP_TRY(cudaEventRecord(hp.freed[b], hp.cs), "event record");
            HP_TRY(cudaEventRecord(hp.done, hp.cs), "event record");
        }
        HP_TRY(cudaStreamWaitEvent(s, hp.done, 0), "stream wait");
        hp.next = b ^ 1;
        hp.chain = s;
        hp.chained = true;
    }
    h->last_launches = nl;
    if (sync) HP_TRY(cudaStreamSynchronize(s), "synchronise");
#undef HP_TRY
    return ok();
}

gm_status apply_forward_host(gm_handle h, const void *m_host, void *d_host, void *stream) {
    return host_apply(h, m_host, d_host, stream, true, true);
}

gm_status apply_transpose_host(gm_handle h, const void *d_host, void *m_host, void *stream) {
    return host_apply(h, d_host, m_host, stream, false, true);
}

gm_status apply_forward_host_async(gm_handle h, const void *m_host, void *d_host, void *stream) {
    return host_apply(h, m_host, d_host, stream, true, false);
}

gm_status apply_transpose_host_async(gm_handle h, const void *d_host, void *m_host, void *stream) {
    return host_apply(h, d_host, m_host, stream, false, false);
}

gm_status grav_mag_destroy(gm_handle h) {
    if (!h) return ok();
    DeviceGuard dg(h->device);
    cudaDeviceSynchronize();
    free_plan(h);
    return ok();
}

gm_status gm_get_info(gm_handle h, gm_info *out) {
    if (!h || !out) return fail(GM_EINVAL, "NULL argument");
    const gm::Geo &g = h->geo;
    out->sx = g.sx; out->sy = g.sy; out->nz = g.nz; out->nx = g.nx; out->ny = g.ny;
    out->fft_nx = g.NPx; out->fft_ny = g.NPy; out->spec_nx = g.Kx;
    out->kind = h->kind; out->precision = h->precision;
    out->n_model = (int64_t)g.nx * g.ny * g.nz;
    out->n_data = (int64_t)g.sx * g.sy;
    out->spectrum_bytes = h->spec_bytes;
    out->workspace_bytes = h->work_bytes;
    out->setup_ms = h->setup_ms;
    out->spectrum_real = h->spec_real ? 1 : 0;
    return ok();
}

gm_status gm_copy_spectrum(gm_handle h, void *host_out, size_t bytes) {
    if (!h || !host_out) return fail(GM_EINVAL, "NULL argument");
    const gm::Geo &g = h->geo;
    const size_t el = h->precision == GM_F32 ? sizeof(float) : sizeof(double);
    const size_t need = 2 * el * (size_t)g.Kx * g.nz * g.NPy;
    if (bytes < need) return fail(GM_EINVAL, "buffer smaller than spec_nx * nz * fft_ny complex values");
    DeviceGuard dg(h->device);
    if (!h->spec_real && h->precision != GM_DF64) {
        cudaError_t e = cudaMemcpy(host_out, h->spec, h->spec_bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "copy spectrum");
        return ok();
    }
    std::vector<unsigned char> tmp(h->spec_bytes);
    cudaError_t e = cudaMemcpy(tmp.data(), h->spec, h->spec_bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "copy spectrum");
    if (h->precision == GM_DF64) {  // pairs of floats h + l -> doubles
        const size_t nv = h->spec_bytes / (2 * sizeof(float));
        std::vector<double> v(nv);
        const float *f = reinterpret_cast<const float *>(tmp.data());
        if (h->spec_real)  // reals {h, l}
            for (size_t i = 0; i < nv; ++i) v[i] = (double)f[2 * i] + (double)f[2 * i + 1];
        else  // complex {re.h, im.h, re.l, im.l}
            for (size_t i = 0; i < nv; i += 2) {
                v[i] = (double)f[2 * i] + (double)f[2 * i + 2];
                v[i + 1] = (double)f[2 * i + 1] + (double)f[2 * i + 3];
            }
        if (h->spec_real)
            expand_real_spectrum<double>(h, v.data(), static_cast<double *>(host_out));
        else
            std::memcpy(host_out, v.data(), sizeof(double) * nv);
        return ok();
    }
    if (h->precision == GM_F64)
        expand_real_spectrum<double>(h, reinterpret_cast<const double *>(tmp.data()), static_cast<double *>(host_out));
    else
        expand_real_spectrum<float>(h, reinterpret_cast<const float *>(tmp.data()), static_cast<float *>(host_out));
    return ok();
}

gm_status gm_cgls(gm_handle h, const void *d_dev, const void *x0_dev, void *x_dev, double alpha, int iters,
                  double *resid_host, void *stream) {
    NvtxScope nv("gm_cgls");
    if (!h) return fail(GM_EINVAL, "handle is NULL");
    if (!d_dev || !x_dev) return fail(GM_EINVAL, "NULL buffer");
    if (iters < 0 || !(alpha >= 0) || !std::isfinite(alpha)) return fail(GM_EINVAL, "iters >= 0 and alpha >= 0 required");
    DeviceGuard dg(h->device);
    h->host_fwd.chained = h->host_tr.chained = false;
    int nl = 0;
    cudaError_t e = gm::run_cgls(h, d_dev, x0_dev, x_dev, alpha, iters, resid_host,
                                 static_cast<cudaStream_t>(stream), &nl);
    h->last_launches = nl;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(GM_ENOMEM, "CGLS scratch allocation failed");
    }
    if (e != cudaSuccess) return cuda_fail(e, "gm_cgls");
    return ok();
}

gm_status gm_cgls_noalloc(gm_handle h, const void *d_dev, const void *x0_dev, void *x_dev, double alpha,
                          int iters, double *resid_host, void *stream) {
    NvtxScope nv("gm_cgls_noalloc");
    if (!h) return fail(GM_EINVAL, "handle is NULL");
    if (!d_dev || !x_dev) return fail(GM_EINVAL, "NULL buffer");
    if (iters < 0 || !(alpha >= 0) || !std::isfinite(alpha)) return fail(GM_EINVAL, "iters >= 0 and alpha >= 0 required");
    const size_t need = gm::noalloc_cgls_need(h, iters), cap = gm::noalloc_scratch_bytes();
    if (need > cap)
        return fail(GM_EINVAL, "gm_cgls_noalloc needs %zu bytes of scratch for this grid and iteration count; "
                               "its fixed array holds %zu (use gm_cgls)", need, cap);
    DeviceGuard dg(h->device);
    h->host_fwd.chained = h->host_tr.chained = false;
    int nl = 0;
    cudaError_t e = gm::run_cgls_noalloc(h, d_dev, x0_dev, x_dev, alpha, iters, resid_host,
                                         static_cast<cudaStream_t>(stream), &nl);
    h->last_launches = nl;
    if (e != cudaSuccess) return cuda_fail(e, "gm_cgls_noalloc");
    return ok();
}

size_t gm_cgls_noalloc_capacity(void) { return gm::noalloc_scratch_bytes(); }

gm_status gm_last_status(void) { return g_last_status; }
const char *gm_last_error(void) { return g_last_msg; }

const char *gm_status_string(gm_status s) {
    switch (s) {
        case GM_OK: return "GM_OK: success";
        case GM_EINVAL: return "GM_EINVAL: invalid argument";
        case GM_ENOMEM: return "GM_ENOMEM: not enough device memory";
        case GM_ECUDA: return "GM_ECUDA: CUDA runtime error";
        case GM_ETIMEOUT: return "GM_ETIMEOUT: a bounded device wait gave up";
        case GM_EDEVICE: return "GM_EDEVICE: device-side check failed";
        case GM_ENODEV: return "GM_ENODEV: no CUDA device";
    }
    return "unknown gm_status";
}

int gm_last_launch_count(gm_handle h) { return h ? h->last_launches.load() : 0; }

gm_status gm_enable_timing(gm_handle h, int capacity) {
    if (!h || capacity < 0) return fail(GM_EINVAL, "bad handle or capacity");
    DeviceGuard dg(h->device);
    cudaDeviceSynchronize();
    free_timing(h);
    if (capacity == 0) return ok();
    h->tev.resize(2 * (size_t)capacity, nullptr);
    h->tkid.resize(capacity, 0);
    for (auto &e : h->tev) {
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) {
            e = nullptr;
            free_timing(h);
            return cuda_fail(err, "cudaEventCreate");
        }
    }
    return ok();
}

int gm_kernel_times(gm_handle h, gm_kernel_time *out, int max_entries) {
    if (!h || !out || max_entries < 0) {
        fail(GM_EINVAL, "bad argument");
        return -1;
    }
    DeviceGuard dg(h->device);
    double tot[gm::K_COUNT] = {0};
    int cnt[gm::K_COUNT] = {0};
    for (int sl = 0; sl < h->tused; ++sl) {
        float ms = 0;
        if (cudaEventSynchronize(h->tev[2 * sl + 1]) != cudaSuccess ||
            cudaEventElapsedTime(&ms, h->tev[2 * sl], h->tev[2 * sl + 1]) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        tot[h->tkid[sl]] += ms;
        cnt[h->tkid[sl]] += 1;
    }
    h->tused = 0;
    int k = 0;
    for (int id = 0; id < gm::K_COUNT && k < max_entries; ++id) {
        if (!cnt[id]) continue;
        std::memset(out[k].name, 0, sizeof(out[k].name));
        std::strncpy(out[k].name, gm::kKernelNames[id], sizeof(out[k].name) - 1);
        out[k].launches = cnt[id];
        out[k].total_ms = tot[id];
        ++k;
    }
    ok();
    return k;
}

}  // extern "C"
