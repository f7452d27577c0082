// gm_plan.h -- host-side plan record and the launchers each translation unit provides.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <string>
#include <atomic>
#include <vector>

#include "../../include/gravmag.h"
#include "gm_common.cuh"

struct gm_plan {
    int device = 0;
    int kind = GM_GRAVITY;
    int precision = GM_F32;
    gm::Geo geo{};
    int pxr = 0, pyr = 0;
    int Nx = 0, Ny = 0;  // linear-convolution supports sx+nx-1, sy+ny-1
    double dx = 0, dy = 0;
    std::vector<double> zplanes;
    double incl_deg = 90, decl_deg = 0, F_nT = 50000;
    double coef[5] = {0, 0, 0, 0, 0};  // magnetic: F/4pi-scaled coefficients of {Lx, Ly, Lz, Ax, Ay}

    // FFT plans (radix lists) and device twiddle tables in the apply precision.
    gm::FftDesc fx{}, fy{};
    void *tw_x = nullptr, *tw_y = nullptr;

    // Spectra [Kx][nz][NPy], complex in the apply precision; or, with spec_real, the real even
    // spectra of the station-centred generator, [Kx][nz][NPy/2 + 1] (see build_spectra).
    void *spec = nullptr;
    size_t spec_bytes = 0;
    bool spec_real = false;

    // Workspace: the large intermediate (forward [Kx][nz][ny], transpose [nz][ny][Kx]) and the
    // small one (forward [sy][Kx], transpose [Kx][sy]).  The forward and the transpose each have
    // their own pair, so that one of each may run at the same time on different streams.
    void *work_big = nullptr, *work_small = nullptr;        // forward
    void *work_big_tr = nullptr, *work_small_tr = nullptr;  // transpose

    // Host-buffer calls of one direction (capi.cu): two model-sized staging buffers used in turn
    // and a data-sized one, an internal stream for the product and one for the host-link copy of
    // the model, and the events that order them.  While consecutive calls come on one caller
    // stream with nothing else of this direction in between (chained), the internal streams run
    // ahead of the caller's stream, so one call's model copy overlaps its neighbours' kernels.
    struct HostPipe {
        void *stage[2] = {nullptr, nullptr};
        void *stage_small = nullptr;
        cudaStream_t ks = nullptr, cs = nullptr;
        cudaEvent_t fork = nullptr, done = nullptr, ready[2] = {nullptr, nullptr}, freed[2] = {nullptr, nullptr};
        int next = 0;
        cudaStream_t chain = nullptr;
        bool chained = false;
    };
    HostPipe host_fwd, host_tr;
    size_t work_bytes = 0;

    // Register-codelet path (apply_fast.cu): used when both FFT lengths have instantiations.
    bool fast = false;
    void *work_part = nullptr;          // [groups][Kx][NPy] partial depth sums of the forward pass
    void *work_counters = nullptr;      // one arrival counter per column group of the forward pass
    int fast_groups_fwd = 1, fast_lpg_fwd = 1;
    int fast_groups_tr = 1, fast_lpg_tr = 1;

    // CGLS scratch, allocated on the first gm_cgls call.
    void *cgls_buf = nullptr;
    size_t cgls_bytes = 0;

    double setup_ms = 0;
    std::atomic<int> last_launches{0};  // written by concurrent forward and transpose calls

    // Optional per-kernel timing: event pairs around each launch (see gm_enable_timing).
    std::vector<cudaEvent_t> tev;   // 2 per slot
    std::vector<int> tkid;          // kernel id per used slot
    int tused = 0;
};

namespace gm {
// Kernel ids for the timing table.
enum KernelId {
    K_FWD_ROWS = 0, K_FWD_COLS = 1, K_FWD_C2R = 2, K_TR_ROWS = 3, K_TR_COLS = 4, K_TR_C2R = 5, K_CGLS_VEC = 6,
    K_FWD_COLS_INV = 7, K_COUNT = 8
};
extern const char *const kKernelNames[K_COUNT];

// Records an event on s: inside a stream capture as an event-record node of the graph (the
// external flag), otherwise as a plain record (the flag is refused outside a capture).
inline void timing_record(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) cs = cudaStreamCaptureStatusNone;
    if (cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else
        cudaEventRecord(e, s);
}

// Opens the NVTX range of one kernel launch (named for the kernel) and, when per-kernel timing is
// enabled, records the "before" event on s; returns the timing slot or -1.  Every call is paired
// with timing_end.
inline int timing_begin(gm_plan *p, cudaStream_t s, int kid) {
    nvtxRangePushA(kKernelNames[kid]);
    if (p->tused >= (int)p->tkid.size()) return -1;
    int slot = p->tused++;
    p->tkid[slot] = kid;
    timing_record(p->tev[2 * slot], s);
    return slot;
}
inline void timing_end(gm_plan *p, cudaStream_t s, int slot) {
    if (slot >= 0) timing_record(p->tev[2 * slot + 1], s);
    nvtxRangePop();
}
}  // namespace gm

namespace gm {

// Radix list of N (8s, then 4, 2, 3, 5, 7); false if N has another prime factor.
bool make_radices(int N, FftDesc &d);

// Twiddle table exp(-2 pi i e / N), e < N, computed on the host in long double
// and rounded to the element type; allocated on the device.
cudaError_t make_twiddles(int N, int precision, void **dev_out);  // table exp(-2 pi i e / N) in a gm_precision

// Set-up: FP64 entries -> generators -> FP64 2-D FFT -> spectra in the plan's precision.
cudaError_t build_spectra(gm_plan *p, cudaStream_t s);

// Register-codelet apply path (apply_fast.cu).
bool fast_path_supported(int NPx, int NPy);
int fast_column_groups(const gm_plan *p);
void fast_plan_groups(gm_plan *p);
cudaError_t launch_forward_fast(gm_plan *p, const void *m, void *d, cudaStream_t s, int *nl);
cudaError_t launch_transpose_fast(gm_plan *p, const void *d, void *m, cudaStream_t s, int *nl);

// Apply launchers (forward: K4-K6, transpose: K7-K9); return the launch count in *nl.
cudaError_t launch_forward(gm_plan *p, const void *m, void *d, cudaStream_t s, int *nl);
cudaError_t launch_transpose(gm_plan *p, const void *d, void *m, cudaStream_t s, int *nl);

// CGLS on the device (cgls.cu).
cudaError_t run_cgls(gm_plan *p, const void *d, const void *x0, void *x, double alpha, int iters,
                     double *resid_host, cudaStream_t s, int *nl);

// Allocation-free CGLS on the fixed scratch array of cgls.cu; its capacity and the bytes a plan needs.
cudaError_t run_cgls_noalloc(gm_plan *p, const void *d, const void *x0, void *x, double alpha, int iters,
                             double *resid_host, cudaStream_t s, int *nl);
size_t noalloc_scratch_bytes();
size_t noalloc_cgls_need(const gm_plan *p, int iters);

}  // namespace gm
