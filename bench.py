"""Benchmark of the fused f+g stream-collide step (MLUPS and % of HBM roofline).

Default workload: D2Q37, FP32 compute and storage, periodic 4096 x 4096 box,
rho = 1 + 1% random Fourier modes, u = 8 random Fourier modes of amplitude
0.02, T = 1, gamma = 1.4, tau_f = 0.55, tau_g = 0.7.  One bench step = one
solve of 200 lattice time steps: init from resident FP64 fields, 200 fused
steps, moments back to resident FP64 fields.  MLUPS counts cell updates of
both populations (cells x 200 per bench step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload periodic2d|periodic2d_f64|periodic3d|sod2d_s16|...]

Prints one JSON line (rank 0).  Under torchrun (N > 1) every rank runs an
independent replica of the workload (the path has no exchange step on one
grid per GPU), so the value is the sum over ranks ("weak" scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lbm_inputs as li  # noqa: E402

L2_BYTES = 129 * 1024 * 1024

# FP64 paths are bound by GB300's FP64 pipe, not by HBM.  Peak: 152 SMs x 2
# FP64 instructions per clock x 2 flop (FMA) x 2.07 GHz = 1.259 TFLOP/s
# (the GPU's nominal 1.25 TFLOP/s FP64 rate).  Flops per cell update of the
# FP64 step from ncu's SASS counters of the plain one-thread-per-cell kernel
# (profiles/step_d2q37_f64_1024.md, profiles/step_d3q107_f64_64.md):
# D2Q37 299 DFMA + 175 DADD + 95 DMUL per cell = 868 flop;
# D3Q107 786 DFMA + 511 DADD + 152 DMUL per cell = 2235 flop.
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07
FP64_FLOPS_PER_CELL = {0: 868, 1: 2235}

WORKLOADS = {
    # name: lattice, prec, shape, gamma, tau_f, tau_g, steps per solve, fields
    "periodic2d": dict(lattice=0, prec="f32", shape=(4096, 4096), gamma=1.4, tau_f=0.55, tau_g=0.7, steps=200,
                       fields="fourier2d",
                       desc="D2Q37 FP32 periodic 4096x4096, 8-mode Fourier fields (seeds 1,2), gamma 1.4, "
                            "tau_f 0.55, tau_g 0.7, 200 steps per solve"),
    "periodic2d_f64": dict(lattice=0, prec="f64", shape=(4096, 4096), gamma=1.4, tau_f=0.55, tau_g=0.7, steps=20,
                           fields="fourier2d",
                           desc="D2Q37 FP64 periodic 4096x4096, same fields, 20 steps per solve"),
    "periodic2d_s16f": dict(lattice=0, prec="f32_s16f", shape=(4096, 4096), gamma=1.4, tau_f=0.55, tau_g=0.7,
                            steps=200, fields="fourier2d",
                            desc="D2Q37 FP32 compute, FP16 deviation storage, periodic 4096x4096, 200 steps"),
    "periodic2d_s16bf": dict(lattice=0, prec="f32_s16bf", shape=(4096, 4096), gamma=1.4, tau_f=0.55, tau_g=0.7,
                             steps=200, fields="fourier2d",
                             desc="D2Q37 FP32 compute, BF16 deviation storage, periodic 4096x4096, 200 steps"),
    "sod2d": dict(lattice=0, prec="f64", shape=(1000, 4), bc=(1, 0), gamma=1.4, tau_f=0.6, tau_g=0.6, steps=500,
                  fields="sod",
                  desc="D2Q37 FP64 Sod shock tube 1000x4 (rho 1|0.125, p 1|0.1, zero-gradient x, periodic y), "
                       "gamma 1.4, tau 0.6, 500 steps per solve"),
    "fd2d": dict(lattice=0, prec="f32", shape=(4096, 4096), gamma=1.4, tau_f=0.55, tau_g=0.7, steps=200,
                 fields="fourier2d", scheme="fd", lam=0.03,
                 desc="D2Q37 FP32 finite-difference variant (Sec. III, third-order upwind, lambda 0.03), periodic "
                      "4096x4096, recipe fields, 200 steps per solve"),
    "fd2d_small": dict(lattice=0, prec="f32", shape=(1024, 1024), gamma=1.4, tau_f=0.55, tau_g=0.7, steps=20,
                       fields="fourier2d", scheme="fd", lam=0.03,
                       desc="D2Q37 FP32 finite-difference variant, periodic 1024x1024 (profiling case), 20 steps"),
    "periodic2d_small": dict(lattice=0, prec="f32", shape=(1024, 1024), gamma=1.4, tau_f=0.55, tau_g=0.7, steps=20,
                             fields="fourier2d",
                             desc="D2Q37 FP32 periodic 1024x1024 (profiling case, 0.6 GB state > L2), 20 steps"),
    "periodic2d_f64_small": dict(lattice=0, prec="f64", shape=(1024, 1024), gamma=1.4, tau_f=0.55, tau_g=0.7,
                                 steps=10, fields="fourier2d",
                                 desc="D2Q37 FP64 periodic 1024x1024 (profiling case), 10 steps"),
    "periodic2d_s16f_small": dict(lattice=0, prec="f32_s16f", shape=(1024, 1024), gamma=1.4, tau_f=0.55,
                                  tau_g=0.7, steps=20, fields="fourier2d",
                                  desc="D2Q37 FP16 storage periodic 1024x1024 (profiling case), 20 steps"),
    "periodic3d_small": dict(lattice=1, prec="f32", shape=(96, 96, 96), gamma=1.4, tau_f=0.6, tau_g=0.6, steps=10,
                             fields="fourier3d",
                             desc="D3Q107 FP32 periodic 96^3 (profiling case, 0.8 GB state > L2), 10 steps"),
    "periodic3d_g13": dict(lattice=1, prec="f32", shape=(256, 256, 256), gamma=1.3, tau_f=0.6, tau_g=0.6,
                           steps=100, fields="fourier3d",
                           desc="D3Q107 FP32 periodic 256^3, same fields, gamma 1.3 (delta = 11/3), tau 0.6, "
                                "100 steps per solve"),
    "periodic3d_f64": dict(lattice=1, prec="f64", shape=(256, 256, 256), gamma=1.4, tau_f=0.6, tau_g=0.6,
                           steps=10, fields="fourier3d",
                           desc="D3Q107 FP64 periodic 256^3, same fields, gamma 1.4, tau 0.6, 10 steps per solve"),
    "periodic3d_f64_small": dict(lattice=1, prec="f64", shape=(64, 64, 64), gamma=1.4, tau_f=0.6, tau_g=0.6,
                                 steps=4, fields="fourier3d",
                                 desc="D3Q107 FP64 periodic 64^3 (profiling case, 0.9 GB state > L2), 4 steps"),
    "periodic3d_wide": dict(lattice=1, prec="f32", shape=(256, 48, 48), gamma=1.4, tau_f=0.6, tau_g=0.6, steps=10,
                            fields="fourier3d",
                            desc="D3Q107 FP32 periodic 256x48x48 (profiling case with the bench's 256-cell rows, "
                                 "1.0 GB state > L2), 10 steps"),
    "periodic3d_s16f_wide": dict(lattice=1, prec="f32_s16f", shape=(256, 48, 48), gamma=1.4, tau_f=0.6,
                                 tau_g=0.6, steps=10, fields="fourier3d",
                                 desc="D3Q107 FP16 storage periodic 256x48x48 (profiling case with the bench's "
                                      "256-cell rows, 0.5 GB state > L2), 10 steps"),
    "periodic3d_s16f_small": dict(lattice=1, prec="f32_s16f", shape=(96, 96, 96), gamma=1.4, tau_f=0.6,
                                  tau_g=0.6, steps=10, fields="fourier3d",
                                  desc="D3Q107 FP16 storage periodic 96^3 (profiling case, 0.4 GB state > L2), "
                                       "10 steps"),
    "periodic3d_s16f": dict(lattice=1, prec="f32_s16f", shape=(256, 256, 256), gamma=1.4, tau_f=0.6, tau_g=0.6,
                            steps=100, fields="fourier3d",
                            desc="D3Q107 FP32 compute, FP16 deviation storage, periodic 256^3, 100 steps per solve"),
    "periodic3d": dict(lattice=1, prec="f32", shape=(256, 256, 256), gamma=1.4, tau_f=0.6, tau_g=0.6, steps=100,
                       fields="fourier3d",
                       desc="D3Q107 FP32 periodic 256^3, 8-mode Fourier rho/u/T (seeds 3,4,5), gamma 1.4, "
                            "tau 0.6, 100 steps per solve"),
}


# ---------------------------------------------------------------------------
def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def make_fields(wl, shape):
    if wl["fields"] == "sod":
        return li.sod_fields(shape[0], shape[1])
    if wl["fields"] == "fourier2d":
        return li.fourier_fields(shape, seed_u=1, seed_rho=2)
    if wl["fields"] == "fourier3d":
        return li.fourier_fields(shape, seed_u=3, seed_rho=4, seed_T=5)
    raise ValueError(wl["fields"])


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# the sources that define each recorded kernel (its code and launch shapes)
KERNEL_SOURCES = {"k_step": ("kernels.cuh", "launch_impl.cuh"),
                  "k_step_fd": ("kernels.cuh", "launch_impl.cuh", "fd_march.cuh")}


def kernel_source_hash(kind="k_step"):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1608_06345_gb300", "csrc")
    for f in KERNEL_SOURCES[kind]:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(key):
    """DRAM bytes per launch of the step kernel from the committed ncu
    summary, or None when the kernel source changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    rec = d.get(key)
    kind = "k_step_fd" if key.startswith("k_step_fd") else "k_step"
    if not rec or rec.get("src_hash") != kernel_source_hash(kind):
        return None
    return rec.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
def cpu_oracle_sample(wl, seconds_target=15.0, min_steps=1):
    """Time the FP64 oracle on a bounded sample of the workload: the same
    recipe on a smaller box (1024^2 in 2D, 96^3 in 3D), steps chosen for
    about `seconds_target` of CPU work.  Returns (MLUPS, cores, description)."""
    from oracle import oracle as ora
    shape = (1024, 1024) if len(wl["shape"]) == 2 else (96, 96, 96)
    rho, u, T = make_fields(wl, shape)
    s = ora.Oracle(wl["lattice"], wl["gamma"], wl["tau_f"], wl["tau_g"], shape)
    s.init(rho, u, T)
    t0 = time.perf_counter()
    s.step(1)
    one = time.perf_counter() - t0
    steps = max(min_steps, int(seconds_target / max(one, 1e-6)))
    t0 = time.perf_counter()
    s.step(steps)
    dt = time.perf_counter() - t0
    N = int(np.prod(shape))
    mlups = N * steps / dt / 1e6
    desc = f"FP64 oracle, {'x'.join(map(str, shape))} periodic box of the same recipe, {steps} steps"
    return mlups, ora.get_threads(), desc


def cpu_oracle_single_core(wl, seconds_target=5.0):
    """The oracle on one host core, on a quarter-size box (512^2 / 48^3) of the
    same recipe.  Returns (MLUPS, description)."""
    from oracle import oracle as ora
    keep = ora.get_threads()
    ora.set_threads(1)
    try:
        shape = (512, 512) if len(wl["shape"]) == 2 else (48, 48, 48)
        rho, u, T = make_fields(wl, shape)
        s = ora.Oracle(wl["lattice"], wl["gamma"], wl["tau_f"], wl["tau_g"], shape)
        s.init(rho, u, T)
        t0 = time.perf_counter()
        s.step(1)
        one = time.perf_counter() - t0
        steps = max(1, int(seconds_target / max(one, 1e-6)))
        t0 = time.perf_counter()
        s.step(steps)
        dt = time.perf_counter() - t0
    finally:
        ora.set_threads(keep)
    return int(np.prod(shape)) * steps / dt / 1e6, f"{'x'.join(map(str, shape))} box, {steps} steps, 1 thread"


def cpu_model():
    """Host CPU model name as lscpu reports it (empty if unavailable)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
    except (OSError, subprocess.SubprocessError):
        return ""
    for line in out.splitlines():
        if line.strip().startswith("Model name"):
            return line.split(":", 1)[1].strip()
    return ""


def run_reference(args, wl):
    """Reference arm: the FP64 CPU oracle, as it stands, on the host cores."""
    world, rank, _ = dist_info()
    if rank != 0:
        return
    from oracle import oracle as ora
    shape = (1024, 1024) if len(wl["shape"]) == 2 else (96, 96, 96)
    rho, u, T = make_fields(wl, shape)
    s = ora.Oracle(wl["lattice"], wl["gamma"], wl["tau_f"], wl["tau_g"], shape)
    s.init(rho, u, T)
    N = int(np.prod(shape))
    steps_per = 2
    for _ in range(args.warmup):
        s.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step(steps_per)
    dt = time.perf_counter() - t0
    mlups = N * steps_per * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": "MLUPS (f+g)", "value": mlups, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["desc"], "sample": f"{'x'.join(map(str, shape))} box, {steps_per} steps per bench step"},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": ora.get_threads(), "kind": "oracle",
                         "sample": f"{'x'.join(map(str, shape))} periodic box of the same recipe, "
                                   f"{steps_per} lattice steps per bench step"},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def run_ours(args, wl):
    import torch
    world, rank, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    device = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(device)
    from paper_1608_06345_gb300 import lbm
    lbm.load()

    prec = lbm.PREC_NAMES[wl["prec"]]
    shape = wl["shape"]
    D = len(shape)
    N = int(np.prod(shape))
    S = wl["steps"]
    rho, u, T = make_fields(wl, shape)

    stream = torch.cuda.current_stream()
    solver = lbm.Solver(wl["lattice"], wl["gamma"], wl["tau_f"], wl["tau_g"], shape, bc=wl.get("bc", (0, 0, 0)),
                        prec=prec, stream=stream)
    if wl.get("scheme") == "fd":
        solver.set_fd_kernel({"auto": lbm.LBM_FD_AUTO, "cell": lbm.LBM_FD_CELL, "march": lbm.LBM_FD_MARCH}[args.fd_kernel])
    d_rho = torch.from_numpy(rho).to(device)
    d_u = torch.from_numpy(np.ascontiguousarray(u)).to(device)
    d_T = torch.from_numpy(T).to(device)
    o_rho = torch.empty_like(d_rho)
    o_u = torch.empty_like(d_u)
    o_T = torch.empty_like(d_T)

    def bench_step(ev_pairs=None):
        solver.init(d_rho, d_u, d_T)
        if ev_pairs is not None:
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
        if wl.get("scheme") == "fd":
            solver.step_fd(S, wl["lam"])
        else:
            solver.step(S)
        if ev_pairs is not None:
            b.record(stream)
            ev_pairs.append((a, b))
        solver.moments_device(o_rho, o_u, o_T)

    def barrier():
        from paper_1608_06345_gb300 import replicas
        replicas.barrier()
        torch.cuda.synchronize()

    # pick the fastest compiled launch shape on this instance (trials write
    # only the idle buffer; the state is untouched)
    from paper_1608_06345_gb300 import autotune
    solver.init(d_rho, d_u, d_T)
    if wl.get("scheme") == "fd":
        tuned = {"index": -1, "stage": 0, "block": 128 if wl["lattice"] == 0 else 64}
    elif args.shape is not None:  # a fixed compiled shape instead of the autotuner's pick (profiling)
        lbm.lbm_set_shape(solver.h, args.shape)
        st, bx = lbm.lbm_shape_info(wl["lattice"], prec, args.shape)
        tuned = {"index": args.shape, "stage": st, "block": bx}
    else:
        tuned = autotune.tune(solver, reps=5, cache_path=None)

    for _ in range(max(args.warmup, 0)):
        bench_step()
    solver.sync()

    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.5)
    step_events = []
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    barrier()
    start.record(stream)
    for _ in range(args.steps):
        bench_step(step_events)
    stop.record(stream)
    barrier()
    clk = clocks.stop() if clocks else None
    solver.sync()  # raises on a non-finite state
    elapsed = start.elapsed_time(stop) / 1e3
    step_kernel_s = sum(a.elapsed_time(b) for a, b in step_events) / 1e3 / (args.steps * S)
    from paper_1608_06345_gb300 import replicas
    elapsed = replicas.max_over_ranks(elapsed, device=device)
    mlups = replicas.job_throughput(N * S * args.steps, elapsed, world) / 1e6

    # end to end through the C ABI with host buffers: pinned fields in,
    # moments out, copies inside the timed region
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    h_rho, h_u, h_T = pin(rho), pin(u.reshape(-1)), pin(T)
    r_rho = torch.empty(N, dtype=torch.float64).pin_memory().numpy()
    r_u = torch.empty(D * N, dtype=torch.float64).pin_memory().numpy()
    r_T = torch.empty(N, dtype=torch.float64).pin_memory().numpy()
    e2e_steps = max(1, min(args.steps, 5))

    def e2e_solve():
        lbm.lbm_init(solver.h, h_rho, h_u, h_T)
        if wl.get("scheme") == "fd":
            lbm.lbm_step_fd(solver.h, S, wl["lam"])
        else:
            lbm.lbm_step(solver.h, S)
        lbm.lbm_moments(solver.h, r_rho, r_u, r_T)

    e2e_solve()  # untimed warm-up of the host-buffer path
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_solve()
    barrier()
    e2e_dt = time.perf_counter() - t0
    e2e_dt = replicas.max_over_ranks(e2e_dt, device=device)
    e2e_mlups = replicas.job_throughput(N * S * e2e_steps, e2e_dt, world) / 1e6

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    word = {"f64": 8, "f32": 4, "f32_s16f": 2, "f32_s16bf": 2}[wl["prec"]]
    cells_per_s = N / step_kernel_s
    Q = 37 if wl["lattice"] == 0 else 107
    bytes_per_cell = 2 * Q * 2 * word
    peak, peak_kind = measured_peaks()
    achieved = N * bytes_per_cell / step_kernel_s / 1e9
    kname = "k_step_fd" if wl.get("scheme") == "fd" else "k_step"
    key = f"{kname}_{'d2q37' if wl['lattice'] == 0 else 'd3q107'}_{wl['prec']}_{'x'.join(map(str, shape))}"
    traffic = recorded_traffic(key)

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, cores, desc = cpu_oracle_sample(wl, seconds_target=args.cpu_seconds)
        v1, desc1 = cpu_oracle_single_core(wl)
        cpu = {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": desc,
               "single_core": {"value": v1, "unit": "MLUPS", "sample": desc1}, "cpu_model": cpu_model(),
               "nproc": os.cpu_count()}

    line = {
        "metric": "MLUPS (f+g)", "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": wl["prec"].split("_")[0], "data": "synthetic",
        "config": {"workload": wl["desc"], "lattice": "D2Q37" if wl["lattice"] == 0 else "D3Q107",
                   "grid": list(shape), "storage": wl["prec"], "lattice_steps_per_bench_step": S,
                   "parallelism": f"replicas x{world}",
                   "l2": f"inputs larger than L2: state {2 * N * 2 * Q * word / 1e9:.1f} GB vs 0.13 GB L2",
                   **({"fd_kernel": args.fd_kernel} if wl.get("scheme") == "fd" else {})},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": key, "bytes_per_cell_update": bytes_per_cell,
                     "step_kernel_us": step_kernel_s * 1e6, "peak_kind": peak_kind,
                     "shape": {"stage": tuned["stage"], "block": tuned["block"], "index": tuned["index"]}},
        "e2e": {"value": e2e_mlups, "unit": "MLUPS", "h2d_bytes_per_step": (2 + D) * N * 8,
                "d2h_bytes_per_step": (2 + D) * N * 8,
                "note": "per bench step = one solve through lbm_init (pinned host fields) + lbm_step + "
                        "lbm_moments (pinned host outputs)"},
        "gpu_launches": args.steps * (S * step_launches(wl, shape) + 2),
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    if wl["prec"] == "f64" and wl["lattice"] in FP64_FLOPS_PER_CELL:
        # the FP64 step is ALU-bound: report it against the FP64 pipe
        fl = FP64_FLOPS_PER_CELL[wl["lattice"]]
        hbm = line["roofline"]
        line["roofline"] = {"bound": "alu", "achieved": fl * cells_per_s / 1e9, "peak": FP64_PEAK_GFLOPS,
                            "unit": "GFLOP/s", "frac": fl * cells_per_s / 1e9 / FP64_PEAK_GFLOPS,
                            "traffic": hbm["traffic"], "kernel": hbm["kernel"], "flops_per_cell_update": fl,
                            "peak_kind": "derived: 152 SMs x 2 FP64 inst/clk x 2 flop x 2.07 GHz",
                            "step_kernel_us": hbm["step_kernel_us"], "hbm_achieved_gbs": hbm["achieved"],
                            "hbm_frac": hbm["frac"], "shape": hbm["shape"]}
    if wl["fields"] == "sod":
        line["us_per_lattice_step"] = elapsed / (args.steps * S) * 1e6
    if world == 1 and args.workload == "periodic2d" and not args.no_configs:
        line["configs"] = {name: measure_config(name, n) for name, n in CONFIG_RUNS}
    if world == 1 and args.workload == "periodic2d" and not args.no_serving:
        line["serving"] = serving_eval(args)
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# The other workloads of the benchmark set, measured in the default run (one
# GPU) so that each has a figure of its own: name -> (workload, lattice steps
# timed).  Each timed region lasts about a second, so that the clock sampler
# sees it; every state but the Sod tube's is far larger than L2.
CONFIG_RUNS = [
    ("periodic3d", 200),        # D3Q107 FP32 256^3, gamma 1.4
    ("periodic3d_g13", 200),    # gamma 1.3
    ("periodic3d_s16f", 400),   # D3Q107 FP16 storage 256^3
    ("periodic2d_s16f", 1400),  # D2Q37 FP16 storage 4096^2
    ("periodic2d_s16bf", 1400), # D2Q37 BF16 storage 4096^2
    ("periodic2d_f64", 60),     # D2Q37 FP64 4096^2 (FP64-pipe bound)
    ("fd2d", 400),              # finite-difference variant 4096^2
    ("sod2d", 100000),          # D2Q37 FP64 Sod 1000x4 (latency bound)
]


def step_launches(wl, shape):
    """Kernel launches per lattice step: a 3D grid with 16-bit storage,
    interior rows and 32-bit byte offsets runs its step as an interior and a
    border launch (FP32 storage as one launch)."""
    if len(shape) != 3 or wl.get("scheme") == "fd" or wl["prec"] != "f32_s16f" and wl["prec"] != "f32_s16bf":
        return 1
    nx, ny, nz = shape
    E = {"f64": 8, "f32": 4, "f32_s16f": 4, "f32_s16bf": 4}[wl["prec"]]
    border = ny * nz - (ny - 6) * (nz - 6)
    return 2 if ny >= 7 and nz >= 7 and nx * ny * nz * E < 2 ** 32 and border <= 65535 else 1


def roofline_of(wl, N, step_s):
    """Roofline record of one step: HBM bytes per cell update 2 Q 2 word
    against the measured copy bandwidth, or for FP64 the flops per cell
    update against the FP64 pipe."""
    word = {"f64": 8, "f32": 4, "f32_s16f": 2, "f32_s16bf": 2}[wl["prec"]]
    Q = 37 if wl["lattice"] == 0 else 107
    bpc = 2 * Q * 2 * word
    peak, peak_kind = measured_peaks()
    hbm = N * bpc / step_s / 1e9
    rec = {"bound": "hbm", "achieved": hbm, "peak": peak, "unit": "GB/s", "frac": hbm / peak,
           "bytes_per_cell_update": bpc, "peak_kind": peak_kind}
    if wl["prec"] == "f64" and wl.get("scheme") != "fd":
        fl = FP64_FLOPS_PER_CELL[wl["lattice"]]
        ach = fl * N / step_s / 1e9
        rec = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
               "frac": ach / FP64_PEAK_GFLOPS, "flops_per_cell_update": fl,
               "peak_kind": "derived: 152 SMs x 2 FP64 inst/clk x 2 flop x 2.07 GHz",
               "hbm_achieved_gbs": hbm, "hbm_frac": hbm / peak}
    return rec


def measure_config(name, lattice_steps):
    """One workload of CONFIG_RUNS on its own instance: autotuned shape, 3
    warm-up lattice steps, then `lattice_steps` steps timed with CUDA events
    on the instance's stream and the SM clocks sampled meanwhile."""
    import torch

    from paper_1608_06345_gb300 import autotune, lbm
    wl = WORKLOADS[name]
    shape = wl["shape"]
    N = int(np.prod(shape))
    dev = torch.device("cuda", torch.cuda.current_device())
    rho, u, T = (torch.from_numpy(np.ascontiguousarray(f)).to(dev) for f in make_fields(wl, shape))
    stream = torch.cuda.current_stream()
    solver = lbm.Solver(wl["lattice"], wl["gamma"], wl["tau_f"], wl["tau_g"], shape, bc=wl.get("bc", (0, 0, 0)),
                        prec=lbm.PREC_NAMES[wl["prec"]], stream=stream)
    solver.init(rho, u, T)
    fd = wl.get("scheme") == "fd"
    tuned = {"index": -1} if fd else autotune.tune(solver, reps=3, cache_path=None)
    step = (lambda n: solver.step_fd(n, wl["lam"])) if fd else solver.step
    # whole solves of the workload's length: the Sod tube and the FD variant
    # stay within the steps where they are defined
    per = min(lattice_steps, wl["steps"])
    step(3)
    solver.sync()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    total, elapsed = 0, 0.0
    while total < lattice_steps:
        solver.init(rho, u, T)  # each timed run is one solve from the initial fields
        torch.cuda.synchronize()
        a.record(stream)
        step(per)
        b.record(stream)
        b.synchronize()
        elapsed += a.elapsed_time(b) / 1e3
        total += per
    clk = clocks.stop()
    solver.sync()  # raises on a non-finite state
    solver.close()
    del rho, u, T
    torch.cuda.empty_cache()
    step_s = elapsed / total
    roof = roofline_of(wl, N, step_s)
    kname = "k_step_fd" if fd else "k_step"
    roof["kernel"] = f"{kname}_{'d2q37' if wl['lattice'] == 0 else 'd3q107'}_{wl['prec']}_{'x'.join(map(str, shape))}"
    roof["traffic"] = recorded_traffic(roof["kernel"])
    rec = {"workload": wl["desc"], "lattice_steps_timed": total, "mlups": N / step_s / 1e6,
           "step_kernel_us": step_s * 1e6, "roofline": roof, "clocks": clk,
           "shape": {k: tuned.get(k) for k in ("index", "stage", "block")}}
    if wl["fields"] == "sod":
        rec["l2"] = "state 2.4 MB fits in L2: a latency-bound case, time per step is its figure"
        rec["us_per_lattice_step"] = step_s * 1e6
    return rec


# ---------------------------------------------------------------------------
def serving_eval(args):
    """Continuous batching of a Poisson stream of shock-tube solves (D2Q37,
    FP32, Nx log-uniform in [256, 16384] x 4, gamma, density/pressure ratios,
    tau and 200-2000 steps drawn per request, seed 6) in a pool with an
    explicit memory budget, against the plain FP64 method (one instance per
    request, one launch per step, served in arrival order).  Returns a dict."""
    from paper_1608_06345_gb300 import lbm, serving
    lbm.load()
    params = li.serving_requests(n=args.serving_requests, seed=6)
    reqs = serving.shock_tube_requests(params)
    budget = args.serving_budget_mb << 20

    def batched(arrivals):
        pool = lbm.Pool(0, lbm.LBM_F32, budget_bytes=budget, max_instances=512, bundle_steps=args.bundle_steps)
        recs = serving.serve(reqs, arrivals, serving.PoolBackend(pool))
        pool.close()
        return recs

    # warm-up (graph instantiation, first launches) on a few requests
    warm = lbm.Pool(0, lbm.LBM_F32, budget_bytes=budget, max_instances=512, bundle_steps=args.bundle_steps)
    serving.serve(reqs[:8], np.zeros(8), serving.PoolBackend(warm))
    warm.close()

    cap_recs = batched(np.zeros(len(reqs)))
    cap = serving.summarize(cap_recs)
    capacity = cap["solves_per_s"]
    loads = []
    for f in (0.5, 0.8, 1.0):
        arr = li.poisson_arrivals(len(reqs), rate=f * capacity, seed=7)
        s = serving.summarize(batched(arr))
        s["offered_load"] = f
        s["rate_per_s"] = f * capacity
        loads.append(s)

    def make_solver(req, prec=lbm.LBM_F64):
        # FP64: whole storage (its default); FP32: the request's reference
        # state, as in the pool, so that the FP32 arms differ in batching only
        ref = dict(rho0=req.rho0, T0=req.T0) if prec == lbm.LBM_F32 else {}
        s = lbm.Solver(0, req.gamma, req.tau_f, req.tau_g, req.shape, bc=req.bc, prec=prec, **ref)
        lbm.lbm_set_graph_steps(s.h, 0)  # the plain method: one launch per step
        return s

    base = base32 = nonfinite = None
    if not args.no_baseline:
        arr = li.poisson_arrivals(len(reqs), rate=0.8 * capacity, seed=7)
        b64_recs = serving.serve_baseline(reqs, arr, make_solver)
        base = serving.summarize(b64_recs)
        base["offered_load_of_batched_capacity"] = 0.8
        b32_recs = serving.serve_baseline(reqs, arr, lambda r: make_solver(r, lbm.LBM_F32))
        base32 = serving.summarize(b32_recs)
        base32["offered_load_of_batched_capacity"] = 0.8
        nonfinite = nonfinite_breakdown(reqs, params, cap_recs, b32_recs, b64_recs, make_solver)
    cells_steps = sum(r.cells * r.steps for r in reqs)
    return {
        "workload": f"{len(reqs)} shock-tube solves, D2Q37 FP32, Nx log-uniform [256, 16384] x 4, gamma "
                    f"U[1.1, 1.67], ratios logU[1, 10], tau U[0.52, 1], steps U[200, 2000], seed 6; pool budget "
                    f"{args.serving_budget_mb} MB, bundle {args.bundle_steps} steps",
        "batched_solves_per_s": capacity, "capacity": cap, "poisson": loads,
        "baseline_fp64_one_per_launch": base,
        "baseline_fp32_one_per_launch": base32,
        "p99_ms_at_0.8": loads[1]["p99_ms"],
        "baseline_p99_ms_at_0.8": base["p99_ms"] if base else None,
        "throughput_vs_baseline": capacity / base["solves_per_s"] if base else None,
        "throughput_vs_fp32_baseline": capacity / base32["solves_per_s"] if base32 else None,
        "nonfinite": nonfinite,
        "cell_updates_requested": cells_steps,
    }


def first_nonfinite_step(req, solver, chunk=10):
    """Lattice step (to `chunk` steps) at which an instance of the request
    first meets a non-finite density or temperature, run alone; None if it
    stays finite."""
    from paper_1608_06345_gb300 import lbm
    solver.init(*req.fields)
    done = 0
    try:
        while done < req.steps:
            n = min(chunk, req.steps - done)
            solver.step(n)
            done += n
            solver.sync()
    except lbm.LbmError as ex:
        if ex.code != lbm.LBM_ENONFINITE:
            raise
        return done
    finally:
        solver.close()
    return None


def nonfinite_breakdown(reqs, params, pool_recs, b32_recs, b64_recs, make_solver):
    """Which requests go non-finite in which arm.  The pooled FP32 instance
    computes bitwise what the same instance computes alone, so the pool and
    the plain FP32 arm must agree request by request.  Requests non-finite
    in FP32 but finite in FP64 are listed with their parameters and the step
    at which the FP32 run first meets a non-finite state (run alone, to 10
    steps); the pool itself stops such an instance at the step where its
    error word is set and reports it at the end of that bundle."""
    from paper_1608_06345_gb300 import lbm
    bad = lambda recs: {r.rid for r in recs if r.status == "nonfinite"}
    p32, s32, s64 = bad(pool_recs), bad(b32_recs), bad(b64_recs)
    by_id = {p["id"]: p for p in params}
    only32 = []
    for req in reqs:
        if req.rid in p32 and req.rid not in s64:
            p = by_id[req.rid]
            only32.append({"id": req.rid, "nx": p["nx"], "gamma": p["gamma"], "tau": p["tau"], "steps": p["steps"],
                           "rho_ratio": p["left"][0] / p["right"][0],
                           "p_ratio": (p["left"][0] * p["left"][2]) / (p["right"][0] * p["right"][2]),
                           "fp32_nonfinite_at_step": first_nonfinite_step(req, make_solver(req, lbm.LBM_F32))})
    # step at which each pooled FP32 failure first meets a non-finite state
    # (run alone, to 10 steps): the device stops the instance there and the
    # host reports it at the end of that bundle, at most bundle_steps later
    pairs = [(first_nonfinite_step(req, make_solver(req, lbm.LBM_F32)), req.steps) for req in reqs
             if req.rid in p32]
    at = [a for a, _ in pairs if a is not None]
    steps = [n for a, n in pairs if a is not None]
    return {"pool_fp32": len(p32), "plain_fp32": len(s32), "plain_fp64": len(s64),
            "pool_equals_plain_fp32": p32 == s32, "fp32_only": only32, "fp64_only": sorted(s64 - p32),
            "fp32_nonfinite_at_step": {"min": min(at) if at else None,
                                       "median": float(np.median(at)) if at else None,
                                       "max": max(at) if at else None,
                                       "median_fraction_of_requested_steps":
                                           float(np.median(np.array(at) / np.array(steps))) if at else None}}


def run_serving(args):
    import torch
    world, rank, local = dist_info()
    torch.cuda.set_device(local if world > 1 else 0)
    sv = serving_eval(args)
    cap = sv["capacity"]
    line = {
        "metric": "batched solves/s", "value": sv["batched_solves_per_s"], "unit": "solves/s", "n_gpus": world,
        "steps": 1, "warmup": 1, "ms_per_step": cap["makespan_s"] * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": sv["workload"]}, "serving": sv,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="periodic2d", choices=sorted(WORKLOADS) + ["serving"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--serving-requests", type=int, default=512)
    ap.add_argument("--serving-budget-mb", type=int, default=256)
    ap.add_argument("--bundle-steps", type=int, default=50)
    ap.add_argument("--no-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving summary of the default line")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads of the default line")
    ap.add_argument("--fd-kernel", default="auto", choices=["auto", "cell", "march"],
                    help="kernel of the finite-difference workloads (lbm_set_fd_kernel)")
    ap.add_argument("--shape", type=int, default=None,
                    help="run this compiled step shape (lbm_shape_info index) instead of autotuning")
    args = ap.parse_args()
    if args.workload == "serving":
        run_serving(args)
        return
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
