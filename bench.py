"""Benchmark of the PSATD tight-focusing path on GB300.

One bench step is one full focal-field job of the f = 1 tight-focus workload on
the 256^3 mapped grid: pulse initialisation on the periodic layer, 378 PSATD
steps to the focus t = R0/c, the 128 x 128 focal-plane sample, and the energy /
divergence diagnostics.  The metric is PSATD cell-steps/s (cells x PSATD steps
per second) and the fraction of the HBM roofline reached by the dominant kernel.
The fields are stored as real float32 (the physical E and B are real; --storage
complex times the complex64 storage instead, and the other storage is reported
beside the headline).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--storage real|complex]

N > 1 runs one independent replica per GPU (the path does not shard); the
value is the total work of all ranks over the slowest rank's time.
--impl reference times the float64 CPU oracle on a bounded sample of the same
workload (one PSATD step on a 256 x 256 x 64 slab of the grid).

Beside the headline (N = 1 only where noted) the line carries: the other field
storage, `e2e` (host buffers through the C ABI), `fp64` (the plain float64
solver, with its arithmetic roofline against the float64 FMA rate measured in
the same run), `focal_forms` (one-shot against stepped focal fields), `batched_sweep`
(64 realisations as one CUDA graph of one-shots), `batched_stepped` (the same 64
realisations stepped to their foci by one persistent launch), `multi_octave` (the 1024^3 float32
multi-octave layer against float64 at 768^3; --multi-octave-steps 0 steps it to
the focus), `surrogate_gemm` (the tensor-core GEMM), `cufft_reference` (cuFFT
through torch.fft as a library reference), `cpu_baseline` (the oracle on one
host core) and `cpu_baseline_all_cores` (one oracle process per host core).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2010_00409_gb300 import replicas as RP  # noqa: E402
from paper_2010_00409_gb300 import workloads as W  # noqa: E402

METRIC = "PSATD cell-steps/s"
UNIT = "cell-steps/s"
STEP_KERNELS = ("fft_x", "fft_y", "fft_z", "kspace_z", "plane_xy")
# algorithmic bytes per cell of one full-field sweep (six components read and written)
SWEEP_BYTES = {"real": 48, "complex": 96}
FALLBACK_HBM_GBS = 6800.0


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-stepped-sweep", action="store_true")
    ap.add_argument("--no-multi-octave", action="store_true")
    ap.add_argument("--no-gemm", action="store_true")
    ap.add_argument("--no-cufft", action="store_true")
    ap.add_argument("--multi-octave-steps", type=int, default=8,
                    help="PSATD steps of the 1024^3 multi-octave run (0: to the focus, then the stepped "
                         "focal field is compared with float64 too)")
    ap.add_argument("--storage", choices=("real", "complex"), default="real")
    ap.add_argument("--jsonl", default=os.environ.get("PSATD_METRICS_LOG"),
                    help="append a condensed record of the run to this JSON-lines file "
                         "(default: $PSATD_METRICS_LOG, else none)")
    a = ap.parse_args()
    a.storage_note = None
    if a.storage == "real" and not real_storage_supported(a.size):
        # the real-field kernels cover 256 x 256 x {64, 128, 256}; the line says so
        a.storage = "complex"
        a.storage_note = ("real storage requested; the real-field kernels cover 256 x 256 x {64, 128, 256} "
                          "grids, so this %d^3 run uses complex storage" % a.size)
    return a


def real_storage_supported(size):
    return size == 256


def dist_env():
    return RP.env()


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of each
# step kernel kind, from one ncu capture at 256^3 (the plane kernels: mean of
# the forward and inverse launches), keyed by (kernel, size, storage); to be
# re-taken whenever that kernel changes.
NCU_TRAFFIC_BYTES = {("plane_xy", 256, "complex"): 1549.25e6, ("plane_xy", 256, "real"): 749.62e6,
                     ("kspace_z", 256, "complex"): 1627.90e6, ("kspace_z", 256, "real"): 824.13e6}
# Where each figure above was captured (profiles/ summaries, one full-set launch each).
NCU_TRAFFIC_SOURCE = {"complex": "profiles/psatd_step_tight_focus_256.md",
                      "real": "profiles/psatd_real_step_tight_focus_256.md"}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", FALLBACK_HBM_GBS)), "measured"
    return FALLBACK_HBM_GBS, "fallback"


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.rows = []
        self.proc = None
        cmd = ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits", "-lms", "200"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for i, nm in enumerate(names):
                if len(r) > 5 + i and r[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- oracle arm
def oracle_sample_rate(size: int, reps: int = 1):
    """One float64 oracle PSATD step on a size x size x size/4 slab of the workload grid."""
    from oracle import psatd_oracle as O
    g, m, p, n_steps, plane = W.tight_focus_workload(N=size)
    nz = max(1, size // 4)
    og = O.Grid(g.Nx, g.Ny, nz, g.dx, g.dy, g.dz, g.x_min, g.y_min, g.z_min, g.c)
    rng = np.random.Generator(np.random.PCG64(0))
    f = rng.standard_normal((6, nz, g.Ny, g.Nx)) + 0j
    dt = (m.R0 / g.c) / n_steps
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        f = O.psatd_step(f, og, dt)
        times.append(time.perf_counter() - t0)
    cells = g.Nx * g.Ny * nz
    return cells, times, "one float64 oracle PSATD step (the oracle's own mixed-radix FFT in numpy, 1 thread) on a %dx%dx%d slab of the %d^3 grid" % (
        g.Nx, g.Ny, nz, size)


def _oracle_worker(size):
    """One spawned process: a warm-up step, then one timed oracle step (seconds)."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    cells, _, _ = oracle_sample_rate(size, reps=1)
    _, times, _ = oracle_sample_rate(size, reps=1)
    return cells, times[0]


def oracle_all_cores_rate(size, procs=None, timeout_s=300):
    """The same oracle sample run as one independent process per host core
    (started with spawn, so none is forked from a process that holds a CUDA
    context); rate = all processes' cells / the slowest process's step time."""
    import multiprocessing as mp
    if procs is None:
        # the cores this process may run on, at most 16, and at most a quarter of the
        # free host memory at ~2.5 GB per process (the 256^3 sample peaks near 2 GB)
        procs = min(len(os.sched_getaffinity(0)), 16)
        free = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
        per = 2.5e9 * (size / 256) ** 3
        procs = max(1, min(procs, int(0.25 * free / per)))
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map_async(_oracle_worker, [size] * procs).get(timeout=timeout_s)
    cells = sum(c for c, _ in res)
    t = max(dt for _, dt in res)
    return {"value": cells / t, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": "%d independent processes, each one float64 oracle PSATD step (1 thread) on a "
                      "%dx%dx%d slab of the %d^3 grid after one warm-up step; rate = their cells / the "
                      "slowest step" % (procs, size, size, max(1, size // 4), size)}


def run_reference(a):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    if a.warmup > 0:
        oracle_sample_rate(a.size, reps=a.warmup)
    cells, times, sample = oracle_sample_rate(a.size, reps=a.steps)
    t = sum(times)
    value = cells * a.steps / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * t / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(a.size, a.storage),
                       **({"storage_note": a.storage_note} if a.storage_note else {})),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    if a.jsonl:
        from paper_2010_00409_gb300 import metrics
        metrics.append(a.jsonl, metrics.bench_record(line))


def workload_config(size, storage="real"):
    g, m, p, n_steps, plane = W.tight_focus_workload(N=size)
    vb = 4 if storage == "real" else 8
    return {"workload": "tight focus f=1, 2-cycle Gaussian at 800 nm, R0=20 lambda, %d^3 mapped grid, "
                        "%d PSATD steps to focus + 128x128 focal plane + diagnostics" % (size, n_steps),
            "grid": [g.Nx, g.Ny, g.Nz], "psatd_steps_per_job": n_steps, "precision": "fp32 storage/arithmetic, "
            "fp64 tables/coordinates/reductions",
            "layout": "SoA [6][Nz][Ny][Nx] " + ("float32 (real fields; half spectrum between kernels)"
                                                if storage == "real" else "complex64"),
            "l2": "inputs larger than L2 (field %.0f MB > 129 MB L2)" % (6 * g.cells * vb / 1e6),
            "parallelism": "replicas"}


# --------------------------------------------------------------------------- our arm
def run_ours(a):
    import torch
    from paper_2010_00409_gb300 import psatd

    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device (the library has no CPU path)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    g, m, p, n_steps, plane = W.tight_focus_workload(N=a.size)
    dt = (m.R0 / g.c) / n_steps
    stream = torch.cuda.Stream(dev)
    ctx = psatd.Context(g, m, dt, 32, stream=stream, real=(a.storage == "real"))
    out_dev = torch.empty((3, plane["nz"], plane["ny"]), dtype=torch.complex64, device=dev)

    def job(c, out):
        c.init_pulse(p)
        c.advance(n_steps)
        c.sample_focal_plane(plane["x_p"], plane["ny"], plane["nz"], plane["y0"], plane["y1"],
                             plane["z0"], plane["z1"], comps=(0, 1, 2), out=out)
        return c.diagnostics()

    for _ in range(a.warmup):
        job(ctx, out_dev)
    ctx.synchronize()

    barrier = RP.barrier

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize(dev)
    t_ms, _, launches, diag = time_jobs(ctx, job, out_dev, a.steps, stream, dev)
    barrier()
    clk = clocks.stop()
    # per-kernel durations: the same jobs again, every launch bracketed by events
    t_prof, prof, _, _ = time_jobs(ctx, job, out_dev, a.steps, stream, dev, profile=True)
    t_max = RP.max_over_ranks(t_ms, device=dev)
    value = RP.whole_job_rate(g.cells * n_steps * a.steps, world, t_max / 1e3)
    peak, peak_src = measured_peaks()
    roof, step_hbm = step_roofline(prof, g, a.storage, a.size, peak, peak_src)
    all_total = sum(v[0] for v in prof.values())
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": t_max / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload_config(a.size, a.storage),
                       **({"storage_note": a.storage_note} if a.storage_note else {})),
        "focal_fields_per_s": world * a.steps / (t_max / 1e3),
        "roofline": dict(roof, region="CUDA events around every launch of the same %d jobs, run right after "
                         "the timed region (%.1f ms/job there; the timed region itself runs without per-kernel "
                         "events, which would serialise the launches)" % (a.steps, t_prof / a.steps)),
        "kernel_share": {k: round(v[0] / all_total, 4) for k, v in sorted(prof.items())},
        "step_hbm": step_hbm,
        "clocks": clk,
        "gpu_launches": launches,
        "diag_last": {"energy": diag["energy"], "max_div_E_rel": diag["max_div_E"] / max(diag["max_E_hat"], 1e-300)},
    }
    # the other field storage, same job, fewer jobs (reported beside the headline)
    other = "complex" if a.storage == "real" else "real"
    if other == "real" and not real_storage_supported(a.size):
        line["real_storage"] = {"unavailable": "the real-field kernels cover 256 x 256 x {64, 128, 256} grids"}
    else:
        with psatd.Context(g, m, dt, 32, stream=stream, real=(other == "real")) as c2:
            job(c2, out_dev)
            c2.synchronize()
            k2 = max(1, min(a.steps, 2))
            t2, _, _, _ = time_jobs(c2, job, out_dev, k2, stream, dev)
            _, prof2, _, _ = time_jobs(c2, job, out_dev, k2, stream, dev, profile=True)
            roof2, hbm2 = step_roofline(prof2, g, other, a.size, peak, peak_src)
        line[other + "_storage"] = {"value": world * g.cells * n_steps * k2 / (t2 / 1e3), "unit": UNIT,
                                    "jobs": k2, "ms_per_job": t2 / k2, "roofline": roof2, "step_hbm": hbm2}

    if not a.no_e2e:
        line["e2e"] = e2e_measure(a, ctx, g, m, p, n_steps, plane, stream, dev, world)
    if not a.no_fp64:
        line["fp64"] = fp64_measure(g, m, p, n_steps, dt, dev, stream)
        line["focal_forms"] = focal_forms(ctx, g, m, p, n_steps, plane, dt, dev, stream, out_dev,
                                          line["fp64"]["ms_per_psatd_step"])
    ctx.close()
    if not a.no_sweep:
        line["batched_sweep"] = sweep_measure(dev, stream)
    if not a.no_stepped_sweep and world == 1:
        line["batched_stepped"] = stepped_sweep_measure(dev, stream)
    if not a.no_multi_octave and world == 1:
        line["multi_octave"] = multi_octave_measure(dev, stream, k=a.multi_octave_steps)
    if not a.no_gemm and world == 1:
        line["surrogate_gemm"] = gemm_measure(dev, stream)
    if not a.no_cufft and world == 1 and a.size == 256:
        line["cufft_reference"] = cufft_measure(dev, stream, g, dt, line)
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cells, times, sample = oracle_sample_rate(a.size, reps=1)
        line["cpu_baseline"] = {"value": cells / times[0], "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": sample}
        try:
            line["cpu_baseline_all_cores"] = oracle_all_cores_rate(a.size)
        except Exception as e:  # reported, never fatal: the GPU figures above stand without it
            line["cpu_baseline_all_cores"] = {"unavailable": "%s: %s" % (type(e).__name__, e)}
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
        if a.jsonl:
            from paper_2010_00409_gb300 import metrics
            metrics.append(a.jsonl, metrics.bench_record(line))


def multi_octave_measure(dev, stream, k=8):
    """The multi-octave workload (400-3200 nm, seeded GDD / TOD, f = 0.5) on its
    full 1024^3 float32 layer (complex storage, 51.5 GB): k PSATD steps timed with
    CUDA events (k = 0: all steps to the focus t = R0/c), the energy drift over
    them, the focal field at t = R0/c by one exact step, and its relative L2
    difference from float64 on a 768^3 grid of the same layer; when the steps
    reach the focus, the stepped focal field is compared with it too."""
    import gc
    import torch
    from paper_2010_00409_gb300 import psatd
    g, m, p, prof, n_steps, plane = W.multi_octave_workload(N=1024, seed=0)
    T = m.R0 / g.c
    pa = (plane["ny"], plane["nz"], plane["y0"], plane["y1"], plane["z0"], plane["z1"])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    to_focus = k <= 0
    if to_focus:
        k = n_steps
    stepped = None
    with psatd.Context(g, m, T / n_steps, 32, stream=stream) as ctx:
        ctx.set_pulse_profile(*prof)
        ctx.init_pulse(p)
        d0 = ctx.diagnostics()
        e0.record(stream)
        ctx.advance(k)
        e1.record(stream)
        d1 = ctx.diagnostics()
        ms_step = e0.elapsed_time(e1) / k
        # two more steps with per-launch events: the kernels of one step
        n0 = ctx.launch_count
        ctx.profile_enable(True)
        ctx.advance(2)
        ctx.synchronize()
        kinds = {kk: {"ms_per_step": v[0] / 2, "launches_per_step": v[1] / 2} for kk, v in ctx.profile_read().items()}
        ctx.profile_enable(False)
        launches = (ctx.launch_count - n0) / 2
        if to_focus:
            stepped = ctx.sample_focal_plane(plane["x_p"], *pa, comps=(0, 1, 2))
        ctx.focal_one_shot(p, T, plane["x_p"], *pa, comps=(0, 1, 2))       # warm-up (tables for T)
        t0 = time.perf_counter()
        f32 = ctx.focal_one_shot(p, T, plane["x_p"], *pa, comps=(0, 1, 2))
        t_one = time.perf_counter() - t0
    gc.collect()
    torch.cuda.empty_cache()
    g2, m2, p2, prof2, n2, plane2 = W.multi_octave_workload(N=768, seed=0)
    with psatd.Context(g2, m2, T / n2, 64, stream=stream) as ctx:
        ctx.set_pulse_profile(*prof2)
        f64 = ctx.focal_one_shot(p2, T, plane2["x_p"], *pa, comps=(0, 1, 2))
    gc.collect()
    torch.cuda.empty_cache()
    extra = {}
    if stepped is not None:
        extra["stepped_focal_rel_l2_err_vs_fp64_768"] = float(np.linalg.norm(stepped - f64) / np.linalg.norm(f64))
    peak, peak_src = measured_peaks()
    path_bytes = 96.0 * launches                       # every launch of this path reads and writes the field once
    hbm = {"graded_bytes_per_cell_step": 288, "achieved_GBps_graded": g.cells * 288 / (ms_step * 1e-3) / 1e9,
           "frac_graded": g.cells * 288 / (ms_step * 1e-3) / 1e9 / peak,
           "path_sweeps_per_step": launches, "path_bytes_per_cell_step": path_bytes,
           "achieved_GBps_path": g.cells * path_bytes / (ms_step * 1e-3) / 1e9,
           "frac_path": g.cells * path_bytes / (ms_step * 1e-3) / 1e9 / peak,
           "peak": peak, "peak_source": peak_src, "kernels": kinds}
    return dict({"grid": [g.Nx, g.Ny, g.Nz], "precision": "fp32, complex storage", "psatd_steps": k,
            "ms_per_psatd_step": ms_step, "cell_steps_per_s": g.cells / (ms_step * 1e-3), "hbm": hbm,
            "energy_drift": d1["energy"] / d0["energy"] - 1,
            "max_div_E_rel": d1["max_div_E"] / max(d1["max_E_hat"], 1e-300),
            "steps_to_focus": n_steps,
            "one_shot_focal_fields_per_s": 1.0 / t_one,
            "focal_rel_l2_err_vs_fp64_768": float(np.linalg.norm(f32 - f64) / np.linalg.norm(f64))}, **extra)


def cufft_measure(dev, stream, g, dt, line, reps=5):
    """Library reference (not a path of this package): cuFFT through torch.fft on
    the same six 256^3 fields — forward plus inverse 3D transforms of complex64
    storage and real-to-complex / complex-to-real transforms of float32 storage —
    and, for the complex step, the Eq. 3-4 rotation as PyTorch elementwise
    operations; timed with CUDA events on the bench's stream."""
    import torch
    N = g.Nx
    out = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    with torch.cuda.stream(stream):
        x = torch.randn(6, N, N, N, device=dev, dtype=torch.complex64)
        out["complex_fwd_inv_ms"] = timed(lambda: torch.fft.ifftn(torch.fft.fftn(x, dim=(1, 2, 3)), dim=(1, 2, 3)))
        # per-mode rotation (C = cos(c|k|dt)/1, S = sin(c|k|dt), unit k) on the spectrum
        kx = (2 * np.pi * np.fft.fftfreq(N, g.dx)).astype(np.float32)
        ky = (2 * np.pi * np.fft.fftfreq(N, g.dy)).astype(np.float32)
        kz = (2 * np.pi * np.fft.fftfreq(N, g.dz)).astype(np.float32)
        KX = torch.tensor(kx, device=dev)[None, None, :]
        KY = torch.tensor(ky, device=dev)[None, :, None]
        KZ = torch.tensor(kz, device=dev)[:, None, None]
        km = torch.sqrt(KX * KX + KY * KY + KZ * KZ)
        inv = torch.where(km > 0, 1.0 / torch.clamp(km, min=1e-30), torch.zeros_like(km))
        nx, ny, nz = KX * inv, KY * inv, KZ * inv
        C = torch.cos(g.c * km * dt).to(torch.complex64)
        S = (1j * torch.sin(g.c * km * dt)).to(torch.complex64)
        X = torch.fft.fftn(x, dim=(1, 2, 3))

        def rotate():
            Ex, Ey, Ez, Bx, By, Bz = X.unbind(0)
            kE = nx * Ex + ny * Ey + nz * Ez
            return torch.stack([C * (Ex - nx * kE) + S * (ny * Bz - nz * By),
                                C * (Ey - ny * kE) + S * (nz * Bx - nx * Bz),
                                C * (Ez - nz * kE) + S * (nx * By - ny * Bx),
                                C * Bx - S * (ny * Ez - nz * Ey),
                                C * By - S * (nz * Ex - nx * Ez),
                                C * Bz - S * (nx * Ey - ny * Ex)])
        out["complex_rotation_torch_ms"] = timed(rotate)
        del X, x
        xr = torch.randn(6, N, N, N, device=dev, dtype=torch.float32)
        out["real_fwd_inv_ms"] = timed(lambda: torch.fft.irfftn(torch.fft.rfftn(xr, dim=(1, 2, 3)), s=(N, N, N),
                                                                dim=(1, 2, 3)))
        del xr
    torch.cuda.empty_cache()
    ours_real = line.get("step_hbm", {}).get("ms_per_psatd_step")
    ours_cplx = line.get("complex_storage", {}).get("step_hbm", {}).get("ms_per_psatd_step")
    out["complex_step_ms"] = out["complex_fwd_inv_ms"] + out["complex_rotation_torch_ms"]
    out["note"] = ("cuFFT forward + inverse alone, before any update, against this package's whole step: "
                   "real %.3f ms vs %.3f ms, complex %.3f ms vs %.3f ms" %
                   (out["real_fwd_inv_ms"], ours_real or float("nan"), out["complex_fwd_inv_ms"],
                    ours_cplx or float("nan")))
    return out


def gemm_measure(dev, stream, n=8192, reps=5):
    """The surrogate's tensor-core GEMM (tcgen05, bf16 operands rounded from
    float32, float32 accumulators in tensor memory) on an n^3 problem and on the
    thin 2^20 x 24 x 64 shape of the surrogate's DFT contractions (column-major C),
    timed alone with CUDA events; the n^3 rate against the measured bf16 peak."""
    import torch
    from paper_2010_00409_gb300 import psatd
    out = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        for name, (M, N, K, col_c) in (("square", (n, n, n, False)), ("thin", (1 << 20, 24, 64, True))):
            A = torch.randn(M, K, device=dev)
            B = torch.randn(K, N, device=dev)
            C = torch.zeros(N, M, device=dev).t() if col_c else torch.zeros(M, N, device=dev)
            for _ in range(2):
                psatd.gemm_bf16(A, B, C, stream=stream)
            e0.record(stream)
            for _ in range(reps):
                psatd.gemm_bf16(A, B, C, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / reps
            out[name] = {"shape": [M, N, K], "ms": ms, "tflops": 2.0 * M * N * K / (ms * 1e-3) / 1e12}
            del A, B, C
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak = None
    if os.path.exists(p):
        with open(p) as fh:
            peak = json.load(fh).get("bf16_tflops")
    out["square"]["roofline"] = {"bound": "tensor", "achieved": out["square"]["tflops"], "peak": peak,
                                 "unit": "TFLOP/s", "frac": out["square"]["tflops"] / peak if peak else None,
                                 "peak_source": "measured burst bf16 (MEASURED_PEAKS.json bf16_tflops)"}
    # bf16 operands in memory, fed by tensor copies (psatd_gemm_bf16_tma): C = A B^T
    with torch.cuda.stream(stream):
        A = torch.randn(n, n, device=dev).to(torch.bfloat16)
        B = torch.randn(n, n, device=dev).to(torch.bfloat16)
        C = torch.empty(n, n, device=dev)
        for _ in range(2):
            psatd.gemm_bf16_tma(A, B, C, stream=stream)
        e0.record(stream)
        for _ in range(reps):
            psatd.gemm_bf16_tma(A, B, C, stream=stream)
        e1.record(stream)
        psatd.gemm_synchronize(stream)
        ms = e0.elapsed_time(e1) / reps
        tf = 2.0 * n ** 3 / (ms * 1e-3) / 1e12
        ref = A[:256].double() @ B[:256].double().t()
        err = float((C[:256, :256].double() - ref).abs().max() / n ** 0.5)
        out["square_bf16_tma"] = {"shape": [n, n, n], "ms": ms, "tflops": tf, "max_abs_err_over_sqrtK": err,
                                  "roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s",
                                               "frac": tf / peak if peak else None,
                                               "peak_source": "measured burst bf16 (MEASURED_PEAKS.json bf16_tflops)"}}
        del A, B, C
    return out


def time_jobs(ctx, job, out_dev, steps, stream, dev, profile=False):
    """Run `steps` jobs between CUDA events on the library stream; with profile,
    every launch is also bracketed by its own pair of events (which serialises
    the launches and costs ~1-3 %).  Returns (ms, per-kernel {name: (ms,
    launches)}, launches of our kernels, last diagnostics)."""
    import torch
    ctx.profile_enable(profile)
    n0 = ctx.launch_count
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    diag = None
    for _ in range(steps):
        diag = job(ctx, out_dev)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    launches = ctx.launch_count - n0
    t_ms = ev0.elapsed_time(ev1)
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    return t_ms, prof, launches, diag


def step_roofline(prof, g, storage, size, peak, peak_src):
    """Roofline of the dominant per-step kernel (algorithmic bytes = one read and
    one write of the six stored components per cell per launch: 48 B real, 96 B
    complex) and the whole-step HBM figure from every step kernel's launches."""
    B = SWEEP_BYTES[storage]
    step_k = {k: v for k, v in prof.items() if k in STEP_KERNELS}
    dom = max(step_k, key=lambda k: step_k[k][0])
    dom_ms, dom_n = step_k[dom]
    bytes_per_launch = B * g.cells
    achieved = bytes_per_launch / (dom_ms / dom_n / 1e3) / 1e9
    sweep_bytes = sum(B * g.cells * v[1] for v in step_k.values())
    step_total = sum(v[0] for v in step_k.values())
    n_full = sum(v[1] for v in step_k.values())
    n_st = step_k.get("kspace_z", (0.0, 0))[1] or max(n_full // 3, 1)     # one k-space launch per step
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)"
            if peak_src == "measured" else "fallback 6.8 TB/s",
            "traffic": NCU_TRAFFIC_BYTES.get((dom, size, storage)),
            "traffic_source": NCU_TRAFFIC_SOURCE[storage] if (dom, size, storage) in NCU_TRAFFIC_BYTES else None,
            "bytes_per_launch": bytes_per_launch,
            "bytes_per_cell_per_launch": B, "avg_launch_ms": dom_ms / dom_n, "launches": dom_n}
    hbm = {"algorithmic_bytes_per_cell_step": sweep_bytes / n_st / g.cells,
           "achieved_GBps": sweep_bytes / (step_total / 1e3) / 1e9,
           "frac_of_measured_peak": sweep_bytes / (step_total / 1e3) / 1e9 / peak,
           "ms_per_psatd_step": step_total / n_st,
           "kernels": {k: {"avg_launch_ms": ms / n, "achieved_GBps": bytes_per_launch / (ms / n / 1e3) / 1e9,
                           "frac": bytes_per_launch / (ms / n / 1e3) / 1e9 / peak,
                           "traffic": NCU_TRAFFIC_BYTES.get((k, size, storage)), "launches": n}
                       for k, (ms, n) in step_k.items() if n > 0}}
    return roof, hbm


def e2e_measure(a, ctx, g, m, p, n_steps, plane, stream, dev, world):
    """The same job through the public API with host buffers: the initial six
    components come from pinned host memory (set_field), the focal plane and the
    diagnostics go back to the host, every step."""
    import torch
    ctx.init_pulse(p)
    host_in = torch.empty((6, g.Nz, g.Ny, g.Nx), dtype=ctx.dtype, pin_memory=True)
    host_in.copy_(ctx.fields.cpu())
    host_out = torch.empty((3, plane["nz"], plane["ny"]), dtype=torch.complex64, pin_memory=True)
    import ctypes as C
    from paper_2010_00409_gb300 import psatd
    L = psatd.lib()

    def step():
        psatd._check(L.psatd_set_field(ctx._ptr, -1, C.c_void_p(host_in.data_ptr()), 0), ctx._ptr)
        ctx.set_time(0.0)
        ctx.advance(n_steps)
        psatd._check(L.psatd_sample_focal_plane(
            ctx._ptr, plane["x_p"], plane["ny"], plane["nz"], plane["y0"], plane["y1"], plane["z0"],
            plane["z1"], 7, C.c_void_p(host_out.data_ptr()), 0), ctx._ptr)
        return ctx.diagnostics()

    step()
    ctx.synchronize()
    k = max(1, min(a.steps, 3))
    t0 = time.perf_counter()
    for _ in range(k):
        step()
    ctx.synchronize()
    t = time.perf_counter() - t0
    return {"value": world * g.cells * n_steps * k / t, "unit": UNIT,
            "h2d_bytes_per_step": host_in.numel() * host_in.element_size(),
            "d2h_bytes_per_step": host_out.numel() * host_out.element_size() + 7 * 8,
            "steps": k, "ms_per_step": 1e3 * t / k}


def fp64_peak_measure(dev, stream, iters=4096, reps=5):
    """Float64 FMA rate of this GPU (TFLOP/s): the library's probe kernel, eight
    independent FMA chains per thread, 8 blocks of 256 threads per SM, timed with
    CUDA events on the launching stream after two warm-up launches."""
    import torch
    from paper_2010_00409_gb300 import psatd
    blocks, threads = 8 * torch.cuda.get_device_properties(dev).multi_processor_count, 256
    out = torch.empty(blocks * threads, dtype=torch.float64, device=dev)
    for _ in range(2):
        psatd.fp64_fma_probe(out, blocks, threads, iters, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        psatd.fp64_fma_probe(out, blocks, threads, iters, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / reps
    assert bool(torch.isfinite(out).all())
    return 16.0 * iters * blocks * threads / (ms * 1e-3) / 1e12


# Executed float64 instructions per cell-step of the 256^3 float64 step (ncu
# sass counters over its five launches: x, y, the fused z pass, y, x), from the
# capture summarised in profiles/fp64_step_256.md; re-take when those kernels
# change.  DADD + DMUL + DFMA thread instructions, and their flops (DFMA = 2).
FP64_EXECUTED_256 = {"instr_per_cell_step": 900.56, "flop_per_cell_step": 1078.84,
                     "fp64_pipe_active_pct": "84.7-86.7", "source": "profiles/fp64_step_256.md"}


def fp64_measure(g, m, p, n_steps, dt, dev, stream, n=10):
    """The plain float64 GPU solver on the same grid: n PSATD steps, with its
    arithmetic roofline.  The float64 pipe issues one DADD, DMUL or DFMA per lane
    per cycle, so the bound is the instruction rate: executed float64
    instructions per cell-step (ncu, FP64_EXECUTED_256) against the probe's rate
    (its flops / 2: DFMA chains).  The nominal-flop figure (5 N log2 N per
    complex transform, forward and inverse, six components, plus 80 for the
    update) is kept beside it."""
    import torch
    from paper_2010_00409_gb300 import psatd
    peak = fp64_peak_measure(dev, stream)
    with psatd.Context(g, m, dt, 64, stream=stream) as c:
        c.init_pulse(p)
        c.advance(2)
        c.synchronize()
        c.profile_enable(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.advance(n)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        prof = c.profile_read()
    flop = 2 * 6 * 5 * math.log2(g.cells) + 80
    rate = g.cells * n / (ms * 1e-3)
    achieved = flop * rate / 1e12
    res = {"value": rate, "unit": UNIT, "psatd_steps": n, "ms_per_psatd_step": ms / n,
           "kernel_ms_per_launch": {k: v[0] / v[1] for k, v in prof.items()},
           "nominal_flop_roofline": {"achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                     "frac": achieved / peak, "flop_per_cell_step": flop}}
    if g.Nx == 256 and g.Ny == 256 and g.Nz == 256:
        ex = FP64_EXECUTED_256
        instr = ex["instr_per_cell_step"] * rate / 1e12
        res["roofline"] = {"bound": "alu", "achieved": instr, "peak": peak / 2, "unit": "T fp64 instr/s",
                           "frac": instr / (peak / 2), "instr_per_cell_step": ex["instr_per_cell_step"],
                           "executed_flop_per_cell_step": ex["flop_per_cell_step"],
                           "executed_TFLOPs": ex["flop_per_cell_step"] * rate / 1e12,
                           "fp64_pipe_active_pct_ncu": ex["fp64_pipe_active_pct"], "counters_from": ex["source"],
                           "peak_source": "measured in this run: float64 FMA chains (psatd_fp64_fma_probe), "
                                          "instructions = flops / 2"}
    else:
        res["roofline"] = dict(res["nominal_flop_roofline"], bound="alu",
                               note="executed-instruction counters were taken at 256^3 only")
    res["roofline"].setdefault("peak_source", "measured in this run: float64 FMA chains (psatd_fp64_fma_probe)")
    return res


def focal_forms(ctx32, g, m, p, n_steps, plane, dt, dev, stream, stepped32, ms_step64, reps=5):
    """Focal fields/s of the stepped FP32 job (just timed), the FP32 and FP64
    one-shot paths (one exact step of T = R0/c, sampled from the spectrum) and the
    plain FP64 stepped solver (from its measured step time), each with the relative
    L2 error of its focal plane against the FP64 one-shot plane."""
    import torch
    from paper_2010_00409_gb300 import psatd
    T = n_steps * dt
    args = (plane["x_p"], plane["ny"], plane["nz"], plane["y0"], plane["y1"], plane["z0"], plane["z1"])
    res = {}
    with psatd.Context(g, m, dt, 64, stream=stream) as c64:
        out64 = torch.empty((3, plane["nz"], plane["ny"]), dtype=torch.complex128, device=dev)
        c64.focal_one_shot(p, T, *args, out=out64)
        c64.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            c64.focal_one_shot(p, T, *args, out=out64)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ref = out64.cpu().numpy()
        res["one_shot_fp64"] = {"focal_fields_per_s": reps / (e0.elapsed_time(e1) / 1e3), "rel_l2_err_vs_fp64": 0.0}
    nref = float(np.linalg.norm(ref))
    res["stepped_fp32"] = {"rel_l2_err_vs_fp64": float(np.linalg.norm(stepped32.cpu().numpy() - ref) / nref)}
    out32 = torch.empty((3, plane["nz"], plane["ny"]), dtype=torch.complex64, device=dev)

    def one_shot_rate(c):
        c.focal_one_shot(p, T, *args, out=out32)
        c.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            c.focal_one_shot(p, T, *args, out=out32)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return {"focal_fields_per_s": reps / (e0.elapsed_time(e1) / 1e3),
                "rel_l2_err_vs_fp64": float(np.linalg.norm(out32.cpu().numpy() - ref) / nref)}

    # the one-shot on both float32 storages: the context's own and the other one
    other_real = not ctx32.real
    key = {True: "one_shot_fp32_real_storage", False: "one_shot_fp32_complex_storage"}
    res[key[ctx32.real]] = one_shot_rate(ctx32)
    if other_real and not (g.Nx == 256 and g.Ny == 256 and g.Nz in (64, 128, 256)):
        res[key[True]] = {"unavailable": "the real-field kernels cover 256 x 256 x {64, 128, 256} grids"}
    else:
        with psatd.Context(g, m, dt, 32, stream=stream, real=other_real) as c2:
            res[key[other_real]] = one_shot_rate(c2)
    res["stepped_fp64_estimate"] = {"focal_fields_per_s": 1e3 / (ms_step64 * n_steps),
                                    "note": "from the measured FP64 PSATD step time x %d steps" % n_steps}
    return res


def sweep_measure(dev, stream, n=64, reps=3, n_check=4):
    """Batched parameter sweep: n seeded realisations (f-number, CEP, ellipticity)
    on uneven mapped grids, each one exact step of T = R0/c to its focal plane,
    all recorded into one CUDA graph and replayed with one launch.  Kernel paths
    and tile widths per grid shape come from the autotuner.  The FP32 focal planes
    of the first n_check realisations are compared with FP64 one-shots."""
    import torch
    from paper_2010_00409_gb300 import psatd
    sweep = W.batched_sweep(n, seed=0)
    t_setup = time.perf_counter()
    items = []
    for g, m, p, T, plane in sweep:
        c = psatd.Context(g, m, T / 100, 32, stream=stream)
        c.autotune(2)
        o = torch.empty((3, plane["nz"], plane["ny"]), dtype=torch.complex64, device=dev)
        args = (plane["x_p"], plane["ny"], plane["nz"], plane["y0"], plane["y1"], plane["z0"], plane["z1"])
        c.focal_one_shot(p, T, *args, out=o)
        items.append((c, p, T, args, o))
    torch.cuda.synchronize(dev)
    t_setup = time.perf_counter() - t_setup
    b = psatd.Batch(stream)
    with b:
        for c, p, T, args, o in items:
            c.focal_one_shot(p, T, *args, out=o)
    b.launch()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        b.launch()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    errs = []
    t64 = 0.0
    for (g, m, p, T, plane), (c, _, _, args, o) in zip(sweep[:n_check], items[:n_check]):
        with psatd.Context(g, m, T / 100, 64, stream=stream) as c64:
            w = c64.focal_one_shot(p, T, *args)
            c64.synchronize()
            q0 = time.perf_counter()
            w = c64.focal_one_shot(p, T, *args)
            t64 += time.perf_counter() - q0
        got = o.cpu().numpy()
        errs.append(float(np.linalg.norm(got - w) / np.linalg.norm(w)))
    shapes = sorted({(g.Nx, g.Ny, g.Nz) for g, *_ in sweep})
    res = {"realisations": n, "grid_shapes": len(shapes), "graph_nodes": b.nodes,
           "focal_fields_per_s": n * reps / (ms / 1e3), "ms_per_graph_launch": ms / reps,
           "setup_s_incl_autotune": t_setup,
           "fp64_one_shot_focal_fields_per_s_eager": n_check / t64 if t64 > 0 else None,
           "max_rel_l2_err_fp32_vs_fp64": max(errs), "err_checked_on": n_check}
    b.close()
    for c, *_ in items:
        c.close()
    return res


def stepped_sweep_measure(dev, stream, n=64, n_check=4, k_steps=4, fp64_boxes=4, fp64_steps=4):
    """The sweep realisations (seeded CEP, ellipticity, f-number; 11 uneven grid
    shapes, 96-192 per axis, complex float32) stepped to their foci: each box is
    initialised on its layer (pulse + projection), ALL boxes are advanced by one
    persistent launch (psatd_multi_advance; box p takes ceil(T_p / dt_C,p) steps
    of T_p / that count, T_p = R0/c), then each focal plane (64 x 64) is
    sampled.  focal_fields_per_s = n / (init + launch + sampling).  Radix
    schedules and tile widths come from psatd_multi_autotune (its time is
    reported apart).  Beside it, over k_steps steps of all boxes: the same boxes
    stepped one context after another (the library's per-box launches), and the
    plain float64 stepped solver on fp64_boxes boxes (whole-job rate scaled from
    fp64_steps timed steps plus its init and sampling).  Errors: float32
    stepped focal planes against float64 one-shots (one exact step of T_p) of
    the first n_check realisations."""
    import torch
    from paper_2010_00409_gb300 import psatd
    sweep = W.batched_sweep(n, seed=0)
    items, steps = [], []
    for g, m, p, T, plane in sweep:
        k = math.ceil(T / g.courant_dt())
        c = psatd.Context(g, m, T / k, 32, stream=stream)
        o = torch.empty((3, plane["nz"], plane["ny"]), dtype=torch.complex64, device=dev)
        args = (plane["x_p"], plane["ny"], plane["nz"], plane["y0"], plane["y1"], plane["z0"], plane["z1"])
        items.append((c, p, args, o))
        steps.append(k)
    ctxs = [it[0] for it in items]
    for c, p, _, _ in items:
        c.init_pulse(p)
    t_tune = time.perf_counter()
    ms_tuned = psatd.multi_autotune(ctxs, 1)
    t_tune = time.perf_counter() - t_tune

    def job():
        for c, p, _, _ in items:
            c.init_pulse(p)
        psatd.multi_advance(ctxs, steps)
        for c, _, args, o in items:
            c.sample_focal_plane(*args, out=o)

    job()
    ctxs[0].synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    job()
    e1.record(stream)
    e1.synchronize()
    ctxs[0].synchronize()                      # no barrier wait expired
    ms_job = e0.elapsed_time(e1)
    errs = []
    for (g, m, p, T, plane), (c, _, args, o) in zip(sweep[:n_check], items[:n_check]):
        with psatd.Context(g, m, T / 100, 64, stream=stream) as c64:
            w = c64.focal_one_shot(p, T, *args)
        errs.append(float(np.linalg.norm(o.cpu().numpy() - w) / np.linalg.norm(w)))
    # per batched step: one persistent launch against per-context launches
    e0.record(stream)
    psatd.multi_advance(ctxs, k_steps)
    e1.record(stream)
    e1.synchronize()
    ms_multi = e0.elapsed_time(e1) / k_steps
    n_launch0 = sum(c.launch_count for c in ctxs)
    e0.record(stream)
    for c in ctxs:
        c.advance(k_steps)
    e1.record(stream)
    e1.synchronize()
    ms_eager = e0.elapsed_time(e1) / k_steps
    eager_launches = (sum(c.launch_count for c in ctxs) - n_launch0) / k_steps
    cells = sum(g.cells for g, *_ in sweep)
    # the plain float64 stepped solver on the first fp64_boxes boxes
    t64 = 0.0
    for (g, m, p, T, plane), k in zip(sweep[:fp64_boxes], steps[:fp64_boxes]):
        with psatd.Context(g, m, T / k, 64, stream=stream) as c64:
            args = (plane["x_p"], plane["ny"], plane["nz"], plane["y0"], plane["y1"], plane["z0"], plane["z1"])
            c64.init_pulse(p)
            c64.advance(1)
            c64.synchronize()
            a0, a1, a2, a3 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
            a0.record(stream)
            c64.init_pulse(p)
            a1.record(stream)
            c64.advance(fp64_steps)
            a2.record(stream)
            c64.sample_focal_plane(*args)
            a3.record(stream)
            a3.synchronize()
            t_step = a1.elapsed_time(a2) / fp64_steps
            t64 += (a0.elapsed_time(a1) + k * t_step + a2.elapsed_time(a3)) / 1e3
    for c in ctxs:
        c.close()
    return {"realisations": n, "grid_shapes": len({(g.Nx, g.Ny, g.Nz) for g, *_ in sweep}),
            "steps_min_max": [min(steps), max(steps)], "cells_total": cells,
            "focal_fields_per_s": n / (ms_job / 1e3), "ms_per_batch_job": ms_job,
            "launches_per_batch_advance": 1,
            "ms_per_batched_step_persistent": ms_multi, "ms_per_batched_step_eager_per_context": ms_eager,
            "eager_launches_per_batched_step": eager_launches,
            "cell_steps_per_s_persistent": cells / (ms_multi / 1e3),
            "autotune_s": t_tune, "autotune_best_ms_per_step": ms_tuned,
            "fp64_stepped_focal_fields_per_s": fp64_boxes / t64,
            "fp64_rate_from": "%d boxes, %d timed steps each scaled to the box's step count" % (fp64_boxes, fp64_steps),
            "max_rel_l2_err_fp32_stepped_vs_fp64_exact": max(errs), "err_checked_on": n_check}


def main():
    a = args_parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
