"""Throughput of the fast BTTB operator: G m and G^T d applies per second.

One step = one forward product d = G m plus one transpose product m' = G^T d
(Algorithm multbttb, t = 1 and t = 2) on the 300 x 250-station, 60-layer
gravity grid with 10 % padding per side (the largest workload that fits one
GPU many times over), FP32 apply, FP64 set-up excluded from the timing as the
paper excludes FFTW planning (Sec. 5, Remark).  Prints one JSON line.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
  python bench.py --table1        # the size sweep of Sec. 5, Table 1 (one JSON line per size)

N > 1 (launched by torch.distributed.run): every rank runs an independent
replica on its own GPU (the operator has no exchange step on one GPU's data);
value = applies of all ranks / the slowest rank's time ("replicas only").

--impl reference times the CPU oracle (dense binary128 prism entries, direct
summation) on bounded samples of the same workload on the host's cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "grav300"
METRIC = "G·m and G^T·d applies/s (FP32 vs FP64 on GPU) at rel err ≤1e-5; % HBM roofline"
UNIT = "applies/s"
FALLBACK_HBM_GBS = 6800.0
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
KERNEL_SOURCES = ["paper_1912_06976_gb300/csrc/gm_fast.cuh", "paper_1912_06976_gb300/csrc/gm_fast_impl.cuh",
                  "paper_1912_06976_gb300/csrc/gm_fft_codelets.cuh", "paper_1912_06976_gb300/csrc/gm_common.cuh",
                  "paper_1912_06976_gb300/csrc/apply_fast.cu"]


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--jsonl", default=None,
                    help="also append each result line, with the run's time, arguments, GPU and host cores, "
                         "to this JSON-lines file")
    ap.add_argument("--table1", action="store_true", help="run the Table 1 size sweep instead")
    ap.add_argument("--table1-k", default="1-12", help="sizes k of the sweep, e.g. 1-12 or 3,6,12")
    ap.add_argument("--table1-stations", type=int, default=16,
                    help="oracle stations sampled per size for the forward error (each is a full row of G)")
    return ap.parse_args(argv)


# ----------------------------------------------------------------------------- ranks
def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def reduce_max_sum(t_ms: float, units: float):
    """(max over ranks of t_ms, sum over ranks of units); identity without a process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return t_ms, units
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    a = torch.tensor([t_ms], dtype=torch.float64, device=dev)
    b = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(a, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return float(a.item()), float(b.item())


def barrier():
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s in sm if mx and s >= 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


# ----------------------------------------------------------------------------- helpers
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, workload: str):
    """dram bytes per launch from the committed ncu summary, if it was taken on the current source."""
    path = os.path.join(ROOT, "profiles", f"dram_traffic_{workload}.txt")
    if not os.path.exists(path):
        return None
    want = kernel_source_hash()
    for ln in open(path):
        if ln.startswith("#") or not ln.strip():
            continue
        f = dict(kv.split("=", 1) for kv in ln.split() if "=" in kv)
        if f.get("kernel") == kernel and f.get("source_sha") == want:
            try:
                return float(f["dram_bytes_per_launch"])
            except (KeyError, ValueError):
                return None
    return None


def cpu_oracle_sample(w, budget_s: float = 12.0, min_batches: int = 1, per_thread: int = 256, seed: int = 1234):
    """Times the oracle on batches of uniformly sampled entries of G (per_thread entries per host
    thread per batch) until the budget is spent, and scales the time per entry to the m*n
    entries one forward or transpose product evaluates (the direct sum's multiply-add per entry
    is negligible next to the entry itself)."""
    import numpy as np

    import oracle as O

    geom = O.Geometry(w.sx, w.sy, w.nz, w.dx, w.dy, w.zplanes, w.pxl, w.pxr, w.pyl, w.pyr, w.kind,
                      w.incl_deg, w.decl_deg, w.F_nT)
    threads = O.threads()
    rng = np.random.default_rng(seed)
    k = threads * per_thread
    done, t_total, batches = 0, 0.0, 0
    while batches < min_batches or t_total < budget_s:
        st = rng.integers(0, w.m, k)
        ce = rng.integers(0, w.n, k)
        t0 = time.perf_counter()
        O.entries(geom, st, ce)
        t_total += time.perf_counter() - t0
        done += k
        batches += 1
    apply_s = t_total / done * w.m * w.n
    return {"value": 1.0 / apply_s, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{done} uniformly sampled entries of G ({t_total:.1f} s, binary128), scaled to the "
                      f"m*n = {w.m * w.n} entries one forward or transpose product evaluates",
            "seconds": t_total}


def cpu_oracle_one_core(w, budget_s: float = 3.0):
    """The same sampled-entry timing of the oracle on one host thread (a shorter sample)."""
    import oracle as O

    n = O.threads()
    O.set_threads(1)
    try:
        r = cpu_oracle_sample(w, budget_s=budget_s, per_thread=256, seed=4321)
    finally:
        O.set_threads(n)
    return {"value_1core": r["value"], "sample_1core": r["sample"]}


def host_cpu():
    """Model name and logical CPU count of the host (lscpu where present)."""
    import platform

    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"model": model or platform.processor() or platform.machine(), "nproc": os.cpu_count() or 1,
            "machine": platform.machine()}


def cpu_fft_baseline(gm, w, budget_s: float = 3.0):
    """The host-CPU FFT baseline on the benchmark workload: the GPU path's algorithm with scipy.fft
    on all host cores (batched R2C over the layers, depth multiply-accumulate, one inverse for G m;
    one forward and n_z inverses for G^T d), on the library's own spectra, FP32 and FP64.  Set-up
    and FFT planning are excluded (Sec. 5); a warm-up apply, then repetitions for about budget_s."""
    import numpy as np

    from paper_1912_06976_gb300 import workloads as W

    workers = os.cpu_count() or 1
    m_np, d_np = W.model(w.name, 0), W.data(w.name, 0)
    out = {"cores": workers, "host": host_cpu(), "library": "scipy.fft (pocketfft) rfft2 / irfft2",
           "algorithm": "same as the GPU path, on the library's spectra"}
    for prec, npdt, name in ((gm.F32, np.float32, "fp32"), (gm.F64, np.float64, "fp64")):
        op = gm.Operator.from_workload(w, precision=prec)
        spec = op.spectrum()
        op.close()
        mm, dd = m_np.astype(npdt), d_np.astype(npdt)
        cpu_fft_apply(spec, w.nz, w.ny, w.nx, w.sy, w.sx, mm, dd, workers)
        times = []
        t_end = time.perf_counter() + budget_s
        while len(times) < 3 or time.perf_counter() < t_end:
            t0 = time.perf_counter()
            cpu_fft_apply(spec, w.nz, w.ny, w.nx, w.sy, w.sx, mm, dd, workers)
            times.append(time.perf_counter() - t0)
        out[name] = {"value": 2.0 / statistics.mean(times), "unit": UNIT, "reps": len(times),
                     "ms_per_step_mean": 1e3 * statistics.mean(times),
                     "ms_per_step_median": 1e3 * statistics.median(times)}
        del spec
    return out


def oracle_dense_timings(names=("grav16", "mag64"), budget_s: float = 2.0):
    """The dense oracle (every entry of a row of G from its prism formula, direct sum) on the two
    small workloads, at one host thread and at all of them: rows of d = G m per second, scaled to
    one forward product (m rows).  A bounded sample of stations per measurement."""
    import numpy as np

    import oracle as O
    from paper_1912_06976_gb300 import workloads as W

    nthreads = O.threads()
    res = {"host": host_cpu(), "arithmetic": f"binary128 ({O.significand_bits()}-bit significand)"}
    for name in names:
        w = W.WORKLOADS[name]
        geom = O.Geometry(w.sx, w.sy, w.nz, w.dx, w.dy, w.zplanes, w.pxl, w.pxr, w.pyl, w.pyr, w.kind,
                          w.incl_deg, w.decl_deg, w.F_nT)
        m = W.model(name, 0)
        row = {"stations": w.m, "cells": w.n}
        for label, th in (("1core", 1), ("all_cores", nthreads)):
            O.set_threads(th)
            try:
                rng = np.random.default_rng(7)
                rows, t = 0, 0.0
                while t < budget_s and rows < w.m:
                    k = min(w.m - rows, th)
                    st = rng.choice(w.m, size=k, replace=False)
                    t0 = time.perf_counter()
                    O.forward(geom, m, stations=st)
                    t += time.perf_counter() - t0
                    rows += k
            finally:
                O.set_threads(nthreads)
            per_product = t / rows * w.m
            row[label] = {"applies_per_s": 1.0 / per_product, "threads": th, "rows_timed": rows,
                          "seconds": t}
        res[name] = row
    return res


# ----------------------------------------------------------------------------- reference arm
def roofline_of(ktimes, inf, step_ms, peak, peak_kind, profiled_traffic_for=None):
    """Roofline record of the dominant kernel (the one with the most device time in `ktimes`,
    {name: (launches, total ms)}): algorithmic bytes per launch over its mean launch time against
    the measured copy rate `peak` (GB/s), and, for the column kernels, 5 N log2 N flops per complex
    transform of length N plus the depth multiply-accumulate against the FP32 peak.  The bound
    reported is the roof that the kernel's arithmetic intensity selects (above the ridge point of
    the two peaks: the ALU roof)."""
    import math

    w_el = 4
    spec_bytes = inf.spectrum_bytes  # as stored: complex, or real even (a quarter) for gravity
    alg = {"fwd_rows_r2c": w_el * inf.n_model, "fwd_cols_mac": spec_bytes, "fwd_cols_inv": 0,
           "fwd_rows_c2r": w_el * inf.n_data, "tr_rows_r2c": w_el * inf.n_data, "tr_cols": spec_bytes,
           "tr_rows_c2r": w_el * inf.n_model}
    dom = max(ktimes, key=lambda k: ktimes[k][1])
    dom_ms = ktimes[dom][1] / ktimes[dom][0]
    achieved = alg[dom] / (dom_ms / 1e3) / 1e9
    traffic = profiled_traffic(dom, profiled_traffic_for) if profiled_traffic_for else None
    apply_bytes = w_el * (inf.n_model + inf.n_data) + spec_bytes  # per forward or transpose product
    fx, fy, kx, nz = inf.fft_nx, inf.fft_ny, inf.spec_nx, inf.nz
    tf_y = 5.0 * fy * math.log2(fy)
    mac = (4.0 if inf.spectrum_real else 8.0) * kx * nz * fy
    col_flops = {"fwd_cols_mac": kx * nz * tf_y + mac + kx * tf_y, "tr_cols": kx * tf_y + mac + kx * nz * tf_y}
    hbm = {"kernel": dom, "achieved_gbs": achieved, "peak_gbs": peak, "frac": achieved / peak,
           "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)", "algorithmic_bytes_per_launch": alg[dom]}
    if dom in col_flops:
        alu = {"kernel": dom, "gflop_per_launch": col_flops[dom] / 1e9,
               "achieved_tflops": col_flops[dom] / (dom_ms / 1e3) / 1e12, "peak_tflops": FP32_PEAK_TFLOPS,
               "frac": col_flops[dom] / (dom_ms / 1e3) / 1e12 / FP32_PEAK_TFLOPS,
               "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"}
    else:
        alu = None
    # With the real even spectrum the column kernels do ~25 flop per algorithmic byte, above the
    # ridge (~12 flop/B), so the FP32 ALU roof is the lower one.
    ridge = FP32_PEAK_TFLOPS * 1e12 / (peak * 1e9)
    intensity = (col_flops[dom] / alg[dom]) if (dom in col_flops and alg[dom]) else 0.0
    common = {"kernel": dom, "traffic": traffic, "algorithmic_bytes_per_launch": alg[dom],
              "spectrum_form": "real even (quarter)" if inf.spectrum_real else "complex",
              "kernel_ms_per_launch": dom_ms, "intensity_flop_per_byte": intensity, "ridge_flop_per_byte": ridge,
              "apply_effective_gbs": 2 * apply_bytes / (step_ms / 1e3) / 1e9,
              "apply_frac_of_hbm": 2 * apply_bytes / (step_ms / 1e3) / 1e9 / peak,
              "kernel_share": {k: v[1] / sum(x[1] for x in ktimes.values()) for k, v in ktimes.items()}}
    if alu is not None and intensity > ridge:
        return {"bound": "alu", "achieved": alu["achieved_tflops"], "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": alu["frac"], "peak_source": alu["peak_source"], **common, "hbm_view": hbm}
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": hbm["peak_source"], **common, "alu_view": alu}


def gpu_name():
    try:
        import torch

        return torch.cuda.get_device_name(0) if torch.cuda.is_available() else None
    except Exception:  # the record is informational
        return None


def emit(line, args):
    """Prints one result line; with --jsonl also appends it, with a record of the run, to that file."""
    print(json.dumps(line), flush=True)
    if getattr(args, "jsonl", None):
        rec = dict(line)
        rec["record"] = {"time_utc": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()), "argv": sys.argv[1:],
                         "gpu": gpu_name(), "host_cores": os.cpu_count()}
        with open(args.jsonl, "a") as f:
            f.write(json.dumps(rec) + "\n")


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1912_06976_gb300 import workloads as W

    w = W.WORKLOADS[args.workload]
    per_thread = 2048  # entries per host thread and step: a few ms of oracle work, so thread start-up is noise
    for k in range(args.warmup):
        cpu_oracle_sample(w, budget_s=0.0, min_batches=1, per_thread=per_thread, seed=k)
    vals, secs = [], 0.0
    for k in range(args.steps):
        r = cpu_oracle_sample(w, budget_s=0.0, min_batches=1, per_thread=per_thread, seed=1000 + k)
        vals.append(r["value"])
        secs += r["seconds"]
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * secs / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f128 (binary128)",
            "data": "synthetic", "config": workload_config(w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                             "sample": f"each step: {per_thread * r['cores']} uniformly sampled entries of G "
                                       f"({per_thread} per thread, binary128), scaled to the m*n entries of one "
                                       f"product"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    emit(line, args)
    return 0


def workload_config(w, info=None):
    cfg = {"workload": f"{w.name}: {'gravity' if w.kind == 0 else 'magnetic'} {w.sx}x{w.sy} stations, "
                       f"{w.nz} layers of {w.dx:g} m cells, padding {w.pxl}/{w.pyl} cells per side",
           "stations": w.m, "cells": w.n, "step": "1 forward + 1 transpose product (2 applies)",
           "apply_precision": "fp32 (fp64 set-up)", "l2": "flushed between steps (256 MiB write, untimed)"}
    if info is not None:
        cfg["fft"] = f"{info.fft_nx}x{info.fft_ny}"
    return cfg


# ----------------------------------------------------------------------------- our arm
def time_steps(op, m, d, outd, outm, flush, steps):
    """Per-step CUDA-event times (ms) of forward + transpose, L2 flushed between steps (eager launches)."""
    import torch

    st = torch.cuda.current_stream()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 0xFF)
        starts[k].record(st)
        op.forward(m, out=outd)
        op.transpose(d, out=outm)
        ends[k].record(st)
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in zip(starts, ends)]


def capture_steps(op, m, d, outd, outm, flush, steps, concurrent=False):
    """One CUDA graph holding `steps` steps (flush, start event, forward, transpose, end event) so
    that the timed replay measures device time without host launch gaps.  With concurrent, each
    step's forward and transpose (independent products; the handle gives each its own workspace)
    run on two streams that fork after the start event and join before the end event.  Returns
    (graph, starts, ends) or None when this torch cannot record timing events inside a graph."""
    import torch

    try:
        starts = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(steps)]
    except TypeError:
        return None
    g = torch.cuda.CUDAGraph()
    cs, ts = torch.cuda.Stream(), torch.cuda.Stream()
    cs.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(g, stream=cs):
        for k in range(steps):
            flush.fill_(k & 0xFF)
            starts[k].record()
            if concurrent:
                ts.wait_stream(cs)
                op.forward(m, out=outd)
                op.transpose(d, out=outm, stream=ts)
                cs.wait_stream(ts)
            else:
                op.forward(m, out=outd)
                op.transpose(d, out=outm)
            ends[k].record()
    torch.cuda.synchronize()
    return g, starts, ends


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1912_06976_gb300 import gravmag as gm
    from paper_1912_06976_gb300 import workloads as W

    w = W.WORKLOADS[args.workload]
    op = gm.Operator.from_workload(w, precision=gm.F32)
    inf = op.info
    m = torch.as_tensor(W.model(w.name, 0), dtype=torch.float32, device="cuda").contiguous()
    d = torch.as_tensor(W.data(w.name, 0), dtype=torch.float32, device="cuda").contiguous()
    outd = torch.empty(op.data_shape, dtype=torch.float32, device="cuda")
    outm = torch.empty(op.model_shape, dtype=torch.float32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    time_steps(op, m, d, outd, outm, flush, max(args.warmup, 3))
    # the headline graph holds no per-kernel timing events (an event between two launches would
    # serialise them fully instead of letting the next kernel's launch overlap the previous tail)
    cap = capture_steps(op, m, d, outd, outm, flush, args.steps, concurrent=True)
    if cap is not None:
        graph, starts, ends = cap
        graph.replay()  # warm replay; the timed replay re-records the same timing events
        torch.cuda.synchronize()
    # the same steps with forward and transpose one after the other on one stream, for reference
    cap_s = capture_steps(op, m, d, outd, outm, flush, args.steps, concurrent=False)
    serial_ms = None
    if cap_s is not None:
        cap_s[0].replay()
        torch.cuda.synchronize()
        cap_s[0].replay()
        torch.cuda.synchronize()
        serial_ms = [a.elapsed_time(b) for a, b in zip(cap_s[1], cap_s[2])]
        del cap_s
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    if cap is not None:
        graph.replay()
        torch.cuda.synchronize()
        per_step = [a.elapsed_time(b) for a, b in zip(starts, ends)]
        timing_mode = ("one CUDA graph of all timed steps (no host launch gaps); each step's forward and "
                       "transpose, independent products, on two streams")
    else:
        per_step = time_steps(op, m, d, outd, outm, flush, args.steps)
        timing_mode = "eager launches"
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    # per-kernel device times from a second graph of the same steps with an event pair per launch
    op.enable_timing(8 * args.steps + 16)
    cap_t = capture_steps(op, m, d, outd, outm, flush, args.steps)
    if cap_t is not None:
        cap_t[0].replay()  # the events of the last replay are the ones read
        torch.cuda.synchronize()
    else:
        time_steps(op, m, d, outd, outm, flush, args.steps)
    ktimes = op.kernel_times()
    op.enable_timing(0)
    per_step_timed = [a.elapsed_time(b) for a, b in zip(cap_t[1], cap_t[2])] if cap_t is not None else None
    t_ms = sum(per_step)
    t_max, applies = reduce_max_sum(t_ms, 2.0 * args.steps)
    value = applies / (t_max / 1000.0)
    gpu_launches = sum(v[0] for v in ktimes.values())
    ms_per_step_with_kernel_events = (sum(per_step_timed) / args.steps) if per_step_timed else None

    roofline = roofline_of(ktimes, inf, t_ms / args.steps, *measured_peaks(), profiled_traffic_for=w.name)

    # end to end through the host-buffer entry points (pinned host memory, copies timed).  Every
    # step copies its model in and its data out (forward, stream 1) and its data in and its model
    # out (transpose, stream 2); the stream-ordered calls let one step's host-link transfers
    # overlap the neighbouring steps' kernels, and the clock stops after the last step's results
    # are in host memory.  For context: the synchronising calls from two host threads, and one
    # after the other from one thread.
    import threading

    mh = m.cpu().pin_memory()
    dh = d.cpu().pin_memory()
    od = torch.empty(op.data_shape, dtype=torch.float32).pin_memory()
    om = torch.empty(op.model_shape, dtype=torch.float32).pin_memory()
    sf, st = torch.cuda.Stream(), torch.cuda.Stream()
    k_e2e = max(5, min(args.steps, 50))

    def e2e_async(k):
        for _ in range(k):
            op.forward_host_async(mh, od, stream=sf)
            op.transpose_host_async(dh, om, stream=st)
        sf.synchronize()
        st.synchronize()

    e2e_async(3)
    barrier()
    t0 = time.perf_counter()
    e2e_async(k_e2e)
    t_e2e = (time.perf_counter() - t0) * 1e3

    def host_loop(fn, src, dst, stream):
        for _ in range(k_e2e):
            fn(src, dst, stream=stream)

    t0 = time.perf_counter()
    th = [threading.Thread(target=host_loop, args=(op.forward_host, mh, od, sf)),
          threading.Thread(target=host_loop, args=(op.transpose_host, dh, om, st))]
    for t_ in th:
        t_.start()
    for t_ in th:
        t_.join()
    t_e2e_threads = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        op.forward_host(mh, od, stream=sf)
        op.transpose_host(dh, om, stream=sf)
    t_e2e_serial = (time.perf_counter() - t0) * 1e3
    te_max, e_app = reduce_max_sum(t_e2e, 2.0 * k_e2e)
    tt_max, _ = reduce_max_sum(t_e2e_threads, 2.0 * k_e2e)
    ts_max, _ = reduce_max_sum(t_e2e_serial, 2.0 * k_e2e)
    e2e = {"value": e_app / (te_max / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": 4 * (inf.n_model + inf.n_data), "d2h_bytes_per_step": 4 * (inf.n_data + inf.n_model),
           "api": "apply_forward_host_async + apply_transpose_host_async (pinned host buffers; the model "
                  "vectors by the copy engines through double-buffered device staging, the data vectors "
                  "in place by the kernels), forward and transpose on two streams, one host thread, "
                  "host clock from the first call to the synchronisation after the last",
           "steps": k_e2e,
           "sync_two_threads_value": e_app / (tt_max / 1e3),
           "serial_value": e_app / (ts_max / 1e3)}

    # precision: FP32 against the FP64 GPU run (whole vectors) and against the oracle samples
    extra = {}
    if not args.no_fp64:
        op64 = gm.Operator.from_workload(w, precision=gm.F64)
        m64 = torch.as_tensor(W.model(w.name, 0), dtype=torch.float64, device="cuda").contiguous()
        d64 = torch.as_tensor(W.data(w.name, 0), dtype=torch.float64, device="cuda").contiguous()
        od64 = torch.empty(op.data_shape, dtype=torch.float64, device="cuda")
        om64 = torch.empty(op.model_shape, dtype=torch.float64, device="cuda")
        time_steps(op64, m64, d64, od64, om64, flush, 2)
        k64 = max(3, min(args.steps, 10))
        t64 = sum(time_steps(op64, m64, d64, od64, om64, flush, k64))
        extra["fp64"] = {"value": 2 * k64 / (t64 / 1e3), "unit": UNIT, "ms_per_step": t64 / k64,
                         "setup_ms": op64.info.setup_ms}
        # double-float: FP64 vectors, arithmetic on FP32 pairs (GB300's FP32 rate is 64x its FP64 rate)
        opdf = gm.Operator.from_workload(w, precision=gm.DF64)
        oddf = torch.empty(op.data_shape, dtype=torch.float64, device="cuda")
        omdf = torch.empty(op.model_shape, dtype=torch.float64, device="cuda")
        time_steps(opdf, m64, d64, oddf, omdf, flush, 2)
        tdf = sum(time_steps(opdf, m64, d64, oddf, omdf, flush, k64))
        opdf.forward(m64, out=oddf)
        opdf.transpose(d64, out=omdf)
        op64.forward(m64, out=od64)
        op64.transpose(d64, out=om64)
        torch.cuda.synchronize()
        extra["df64"] = {"value": 2 * k64 / (tdf / 1e3), "unit": UNIT, "ms_per_step": tdf / k64,
                         "arithmetic": "pairs of FP32 values (48-bit significand), FP64 vectors",
                         "rel_err_vs_fp64": {
                             "forward": gm.rel_err(oddf.cpu().numpy(), od64.cpu().numpy()),
                             "transpose": gm.rel_err(omdf.cpu().numpy(), om64.cpu().numpy())}}
        op.forward(m, out=outd)
        op.transpose(d, out=outm)
        torch.cuda.synchronize()
        extra["rel_err_fp32_vs_fp64"] = {
            "forward": gm.rel_err(outd.double().cpu().numpy(), od64.cpu().numpy()),
            "transpose": gm.rel_err(outm.double().cpu().numpy(), om64.cpu().numpy())}
        gpath = os.path.join(ROOT, "tests", "golden", f"sampled_{w.name}.json")
        if os.path.exists(gpath):
            g = json.load(open(gpath))
            extra["rel_err_vs_oracle_samples"] = {
                "fp32_forward": gm.rel_err(outd.double().cpu().numpy().ravel()[g["forward_stations"]], g["forward"]),
                "fp32_transpose": gm.rel_err(outm.double().cpu().numpy().ravel()[g["transpose_cells"]],
                                             g["transpose"]),
                "fp64_forward": gm.rel_err(od64.cpu().numpy().ravel()[g["forward_stations"]], g["forward"]),
                "fp64_transpose": gm.rel_err(om64.cpu().numpy().ravel()[g["transpose_cells"]], g["transpose"]),
                "df64_forward": gm.rel_err(oddf.cpu().numpy().ravel()[g["forward_stations"]], g["forward"]),
                "df64_transpose": gm.rel_err(omdf.cpu().numpy().ravel()[g["transpose_cells"]], g["transpose"])}
        op64.close()
        opdf.close()
    # Tikhonov CGLS (alpha = 1e-2, 50 iterations) on the 128 x 128 x 32 magnetic grid: device time
    # per iteration (one G and one G^T product plus the vector updates and FP64 reductions)
    if rank == 0:
        wc = W.WORKLOADS["mag128"]
        opc = gm.Operator.from_workload(wc, precision=gm.F32)
        dc = opc.forward(torch.as_tensor(W.model("mag128", 0), dtype=torch.float32, device="cuda").contiguous())
        xc = torch.empty(opc.model_shape, dtype=torch.float32, device="cuda")
        opc.cgls(dc, 1e-2, 50, out=xc, residuals=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            opc.cgls(dc, 1e-2, 50, out=xc, residuals=False)
        e1.record()
        torch.cuda.synchronize()
        per_it = e0.elapsed_time(e1) / (3 * 50)
        extra["cgls_mag128"] = {"ms_per_iteration": per_it, "iterations": 50, "alpha": 1e-2,
                                "apply_equivalent_per_s": 2.0 / (per_it / 1e3),
                                "fft": f"{opc.info.fft_nx}x{opc.info.fft_ny}"}
        opc.close()
    if serial_ms:
        extra["serial"] = {"value": 2.0 * len(serial_ms) / (sum(serial_ms) / 1e3), "unit": UNIT,
                           "ms_per_step": sum(serial_ms) / len(serial_ms),
                           "timing": "the same graph with forward and transpose on one stream"}
    extra["setup_ms"] = inf.setup_ms
    extra["kernel_ms_per_step"] = {k: v[1] / args.steps for k, v in ktimes.items()}
    extra["ms_per_step_with_kernel_events"] = ms_per_step_with_kernel_events

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(w)
        cpu.pop("seconds", None)
        cpu.update(cpu_oracle_one_core(w))
        cpu["host"] = host_cpu()
        extra["cpu_fft"] = cpu_fft_baseline(gm, w)
        extra["oracle_dense"] = oracle_dense_timings()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps,
                "ms_per_step_median": statistics.median(per_step), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {**workload_config(w, inf), "parallelism": f"replicas{world}" if world > 1 else "1 GPU",
                           "timing": timing_mode},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
                "clocks": clk, "gpu": gpu_name(), **extra}
        emit(line, args)
    op.close()
    if world > 1:
        dist.destroy_process_group()
    del np
    return 0


# ----------------------------------------------------------------------------- Table 1 sweep
def table1_workloads(ks):
    """Sec. 5, Table 1: s_x = 25 k, s_y = 15 k, n_z = 2 k (k = 1..12), without padding and with 5 %
    of the stations per side rounded half up (the n column of Table 1: 918 = 27 x 17 x 2 for k = 1,
    7616 = 56 x 34 x 4 for k = 2).  The table gives no cell size: 25 m cubes here."""
    from paper_1912_06976_gb300 import workloads as W

    out = []
    for k in ks:
        for pad in (0.0, 0.05):
            sx, sy, nz = 25 * k, 15 * k, 2 * k
            px, py = int(pad * sx + 0.5), int(pad * sy + 0.5)
            out.append((k, pad, W.Workload(f"t1_k{k}_p{int(pad * 100)}", W.GRAVITY, sx, sy, nz, 25.0, 25.0, 25.0,
                                           px, py)))
    return out


def cpu_fft_apply(spec, nz, ny, nx, sy, sx, m, d, workers):
    """The host-CPU FFT baseline: the same algorithm as the GPU path with scipy.fft on all host
    cores, using the library's spectra spec[kx][r][ky] (batched R2C over the layers, the depth
    multiply-accumulate, one inverse for G m; one forward and n_z inverses for G^T d)."""
    import numpy as np
    import scipy.fft as sf

    Kx, _, NPy = spec.shape
    NPx = 2 * (Kx - 1)
    S = np.ascontiguousarray(np.transpose(spec, (1, 2, 0)))  # [r][ky][kx]
    x = np.zeros((nz, NPy, NPx), dtype=m.dtype)
    x[:, :ny, :nx] = m
    M = sf.rfft2(x, workers=workers)
    D = np.einsum("rij,rij->ij", S, M)
    fwd = sf.irfft2(D, s=(NPy, NPx), workers=workers)[:sy, :sx]
    y = np.zeros((NPy, NPx), dtype=d.dtype)
    y[:sy, :sx] = d
    Dh = sf.rfft2(y, workers=workers)
    tr = sf.irfft2(np.conj(S) * Dh[None], s=(NPy, NPx), workers=workers)[:, :ny, :nx]
    return fwd, tr


def run_table1(args):
    """For every Table 1 size: GPU FP32 / FP64 applies per second (CUDA graph of forward +
    transpose steps, L2 flushed between steps), the error against the oracle at sampled stations
    and cells, the host-CPU FFT baseline and the dense oracle's rate on the host cores."""
    import numpy as np
    import torch

    import oracle as O
    from paper_1912_06976_gb300 import gravmag as gm
    from paper_1912_06976_gb300 import workloads as W

    if "-" in args.table1_k:
        a, b = (int(v) for v in args.table1_k.split("-"))
        ks = list(range(a, b + 1))
    else:
        ks = [int(v) for v in args.table1_k.split(",")]
    workers = os.cpu_count() or 1
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for k, pad, w in table1_workloads(ks):
        geom = O.Geometry(w.sx, w.sy, w.nz, w.dx, w.dy, w.zplanes, w.pxl, w.pxr, w.pyl, w.pyr, w.kind,
                          w.incl_deg, w.decl_deg, w.F_nT)
        m_np = W.gaussian_random_field(np.random.default_rng(k), w.model_shape, 4.0, 0.2)
        d_np = W.random_vector(w.data_shape, k)
        row = {"table1_k": k, "padding": pad, "stations": [w.sx, w.sy], "nz": w.nz, "cells": w.n}
        rng = np.random.default_rng(100 + k)
        st = np.sort(rng.choice(w.m, size=min(args.table1_stations, w.m), replace=False))
        ce = np.sort(rng.choice(w.n, size=64, replace=False))
        ref_f = O.forward(geom, m_np, stations=st)
        ref_t = O.transpose(geom, d_np, cells=ce)
        for prec, dt, name in ((gm.F32, torch.float32, "fp32"), (gm.F64, torch.float64, "fp64")):
            op = gm.Operator.from_workload(w, precision=prec)
            m = torch.as_tensor(m_np, dtype=dt, device="cuda").contiguous()
            d = torch.as_tensor(d_np, dtype=dt, device="cuda").contiguous()
            outd = torch.empty(op.data_shape, dtype=dt, device="cuda")
            outm = torch.empty(op.model_shape, dtype=dt, device="cuda")
            time_steps(op, m, d, outd, outm, flush, 3)
            steps = 20
            cap = capture_steps(op, m, d, outd, outm, flush, steps)
            if cap is not None:
                g, starts, ends = cap
                g.replay()
                torch.cuda.synchronize()
                g.replay()
                torch.cuda.synchronize()
                per = [a.elapsed_time(b) for a, b in zip(starts, ends)]
            else:
                per = time_steps(op, m, d, outd, outm, flush, steps)
            op.forward(m, out=outd)
            op.transpose(d, out=outm)
            torch.cuda.synchronize()
            f = outd.double().cpu().numpy()
            t = outm.double().cpu().numpy()
            inf = op.info
            row[name] = {"applies_per_s": 2 * steps / (sum(per) / 1e3), "ms_per_apply": sum(per) / (2 * steps),
                         "rel_err_forward": gm.rel_err(f.ravel()[st], ref_f),
                         "rel_err_transpose": gm.rel_err(t.ravel()[ce], ref_t),
                         "fft": [inf.fft_nx, inf.fft_ny], "path": "codelet" if inf.fft_nx in (
                             32, 48, 64, 80, 96, 112, 128, 140, 160, 192, 224, 256, 288, 320, 384, 448, 512, 560, 576,
                             640, 672, 768, 896, 1024) else "generic", "setup_ms": inf.setup_ms}
            # host-CPU FFT baseline on the same spectra and inputs, same precision
            spec = op.spectrum()
            npdt = np.float64 if prec == gm.F64 else np.float32
            mm, dd = m_np.astype(npdt), d_np.astype(npdt)
            cpu_fft_apply(spec, w.nz, w.ny, w.nx, w.sy, w.sx, mm, dd, workers)
            reps, t0 = 0, time.perf_counter()
            while reps < 3 or time.perf_counter() - t0 < 1.0:
                cf, ct = cpu_fft_apply(spec, w.nz, w.ny, w.nx, w.sy, w.sx, mm, dd, workers)
                reps += 1
            cpu_s = (time.perf_counter() - t0) / reps
            row[name]["cpu_fft"] = {"applies_per_s": 2 / cpu_s, "cores": workers,
                                    "rel_err_vs_gpu": max(gm.rel_err(cf, f), gm.rel_err(ct, t))}
            op.close()
        # dense oracle: sampled columns of G^T d, scaled to m * n entries per product
        cells, t_or = 0, 0.0
        while t_or < 1.0:
            idx = rng.choice(w.n, size=O.threads(), replace=False)
            t0 = time.perf_counter()
            O.transpose(geom, d_np, idx)
            t_or += time.perf_counter() - t0
            cells += len(idx)
        row["oracle_dense"] = {"applies_per_s": 1.0 / (t_or / (cells * w.m) * w.m * w.n), "cores": O.threads()}
        emit(row, args)
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.table1:
        return run_table1(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
