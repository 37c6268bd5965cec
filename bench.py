"""Benchmark of the PMACE hot path on GB300: patch-updates/s.

A step is one PMACE iteration (Algorithm 1) over every window of the
workload: the fused agent sweep (steps S0-S5) and the consensus gather (S6),
two kernel launches.  The default workload is a 600 x 600 complex object,
a 256 x 256 probe and an 18 x 18 jittered raster (324 windows) with FP32
amplitudes at Poisson peak 1e5, drawn by the seeded generator (synthetic
stand-in for the paper's LANL image and probe, which are not available).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line is printed by rank 0.  Under torchrun every rank runs an
independent replica of the job on its own GPU (no data-path collective;
"scaling": "weak"); the time is the maximum over ranks.  `--impl reference`
times the FP64 CPU oracle instead (rank 0 only), on a bounded sample of the
same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PMACE patch-updates/s"
UNIT = "patch-updates/s"
ALPHA, RHO, KAPPA = 0.5, 0.5, 1.25
WORKLOAD = ("p256: object 600x600 complex64, probe 256x256 (Gaussian sigma 48 px, random quadratic "
            "phase), 18x18 raster step 20 px +-2 px jitter = 324 windows, FP32 amplitudes, "
            "Poisson peak 1e5, alpha 0.5, rho 0.5, kappa 1.25")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "agent_p256_traffic.json")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2111_14240_gb300", "csrc", f)
                  for f in ("agent.cuh", "agent_xpose.cuh", "cache_hints.cuh", "tmem.cuh", "fft_smem.cuh",
                            "pmace_internal.h")]


def kernel_hash() -> str:
    """Hash of the agent kernels' source code with comments and blank space
    removed, so that a comment edit does not orphan the stored counters."""
    import re
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(p) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(re.sub(r"\s+", "", src).encode())
    return h.hexdigest()[:16]


def agent_bytes_per_patch(np_: int, amp_bytes: int = 4) -> int:
    """Algorithmic HBM bytes of the agent sweep per window: read q, read y,
    write u, write q (complex64 = 8 B, amplitude 4 or 2 B per pixel).  The
    window of the consensus image it reads is L2-resident and not counted."""
    return np_ * np_ * (8 + amp_bytes + 8 + 8)


def iteration_bytes(np_: int, J: int, n1: int, n2: int, amp_bytes: int = 4) -> int:
    """Algorithmic bytes of one whole iteration: the agent sweep plus the
    gather's read of u and its image traffic (write xbar, read Lambda^-1)."""
    return J * (agent_bytes_per_patch(np_, amp_bytes) + np_ * np_ * 8) + n1 * n2 * (8 + 4)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    """One process per GPU under torchrun (RANK/LOCAL_RANK/WORLD_SIZE/MASTER_*
    from the environment).  NCCL when CUDA is available, else gloo;
    PMACE_DIST_BACKEND overrides.  Returns (dist or None, world, rank, local)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = os.environ.get("PMACE_DIST_BACKEND") or ("nccl" if torch.cuda.is_available() else "gloo")
        if not dist.is_initialized():
            dist.init_process_group(backend=backend)
        return dist, world, rank, local
    return None, 1, 0, local


def max_over_ranks(dist, values):
    """Element-wise maximum of a list of floats over all ranks (identity
    without a process group); the only collective of the benchmark."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def weak_scaling_value(world: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput: every rank processes the same work (replicas),
    timed by the slowest rank."""
    return world * units_per_rank / seconds


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def agent_kernel_name(plan) -> str:
    """The agent sweep kernel a plan launches (transposing exchange or in-place cross-CTA stage)."""
    return "agent_xpose_kernel" if plan.get("exchange") else "agent_kernel"


def stored_traffic():
    if not os.path.exists(TRAFFIC_FILE):
        return None
    with open(TRAFFIC_FILE) as f:
        d = json.load(f)
    if d.get("kernel_hash") != kernel_hash():
        return None
    return float(d["bytes_per_launch"])


# --------------------------------------------------------------------- oracle
def oracle_rate(w, seconds: float, max_windows: int | None = None):
    """FP64 oracle on a sub-scan of the workload: Algorithm 1 over the first
    m windows (m sized so one iteration takes about `seconds`).  Returns
    (patch-updates/s, m, iterations timed, seconds)."""
    from oracle import pmace_oracle as orc
    probe, offs, y = w.probe, w.offsets, w.y
    # estimate the per-window cost on a few windows
    m0 = min(8, len(offs))
    t0 = time.perf_counter()
    orc.pmace(y[:m0], probe, offs[:m0], w.x.shape, alpha=ALPHA, rho=RHO, kappa=KAPPA, n_iter=1)
    per = (time.perf_counter() - t0) / m0
    m = max(1, min(len(offs), int(seconds / max(per, 1e-6))))
    if max_windows:
        m = min(m, max_windows)
    t0 = time.perf_counter()
    orc.pmace(y[:m], probe, offs[:m], w.x.shape, alpha=ALPHA, rho=RHO, kappa=KAPPA, n_iter=1)
    dt = time.perf_counter() - t0
    return m / dt, m, dt


def run_reference(args):
    dist, world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    from paper_2111_14240_gb300 import datagen
    w = datagen.make_workload("p256", seed=1)
    J = w.J
    budget = 150.0
    per_step = max(0.2, min(6.0, budget / max(1, args.steps + args.warmup)))
    if args.ref_seconds > 0:
        per_step = args.ref_seconds
    from oracle import pmace_oracle as orc
    probe, offs, y = w.probe, w.offsets, w.y
    m0 = 8
    t0 = time.perf_counter()
    orc.pmace(y[:m0], probe, offs[:m0], w.x.shape, alpha=ALPHA, rho=RHO, kappa=KAPPA, n_iter=1)
    per = (time.perf_counter() - t0) / m0
    m = max(1, min(J, int(per_step / per)))
    sub = (y[:m], probe, offs[:m], w.x.shape)
    v = None
    for _ in range(args.warmup):
        v = orc.pmace(*sub, alpha=ALPHA, rho=RHO, kappa=KAPPA, n_iter=1, v0=v)["v"]
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v = orc.pmace(*sub, alpha=ALPHA, rho=RHO, kappa=KAPPA, n_iter=1, v0=v)["v"]
    dt = time.perf_counter() - t0
    val = m * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"Algorithm 1 (FP64 numpy, single thread) over the first {m} of "
                                   f"{J} windows per step; each step one iteration"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------- ours
def run_ours(args):
    import torch
    dist, world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    from paper_2111_14240_gb300 import datagen
    from paper_2111_14240_gb300 import pmace as pm

    w = datagen.make_workload("p256", seed=1)
    J, np_ = w.J, w.np_
    n1, n2 = w.x.shape
    probe32 = np.ascontiguousarray(w.probe.astype(np.complex64))
    y32 = np.ascontiguousarray(w.y.astype(np.float32))
    stream = torch.cuda.current_stream()

    rec = pm.Reconstruction(probe32, w.offsets, y32, (n1, n2), kappa=KAPPA, stream=stream)
    plan = rec.plan()
    rec.iterate(args.warmup, ALPHA, RHO)
    torch.cuda.synchronize()
    pm.pmace_set_profiling(rec.h, True)
    pm.pmace_kernel_times(rec.h, reset=True)

    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        start.record(stream)
        rec.iterate(args.steps, ALPHA, RHO)
        stop.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = start.elapsed_time(stop)
    kt = pm.pmace_kernel_times(rec.h, reset=True)
    pm.pmace_set_profiling(rec.h, False)
    r_fp, r_data = rec.residual()
    rec.close()

    # end to end through the C ABI from pinned host buffers: create (H2D of
    # probe, offsets, amplitudes), K iterations, residual and image (D2H)
    y_pin = torch.from_numpy(y32).pin_memory()
    p_pin = torch.view_as_real(torch.from_numpy(probe32)).contiguous().pin_memory()
    img_pin = torch.empty((n1, n2, 2), dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    h = pm.pmace_create(n1, n2, np_, J, KAPPA, p_pin, w.offsets, y_pin, pm.PMACE_AMP_F32,
                        inputs_on_device=False, stream=stream)
    pm.pmace_iterate(h, args.steps, ALPHA, RHO, stream=stream)
    pm.pmace_residual(h, stream=stream)
    pm.pmace_get_image(h, img_pin, stream=stream)
    e2e_s = time.perf_counter() - t0
    pm.pmace_destroy(h)
    h2d = y32.nbytes + probe32.nbytes + w.offsets.nbytes
    d2h = img_pin.numel() * 4 + 16

    ms, e2e_s = max_over_ranks(dist, [ms, e2e_s])
    if rank != 0:
        return 0

    value = weak_scaling_value(world, J * args.steps, ms / 1e3)
    peak, peak_kind = measured_peaks()
    agent_avg_ms = kt["agent_ms"] / max(1, kt["agent_launches"])
    cons_avg_ms = kt["consensus_ms"] / max(1, kt["consensus_launches"])
    bytes_launch = J * agent_bytes_per_patch(np_)
    achieved = bytes_launch / (agent_avg_ms / 1e3) / 1e9
    it_bytes = iteration_bytes(np_, J, n1, n2)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "windows": J, "probe": np_, "image": [n1, n2],
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "no flush: per-step working set (q, u, y) is "
                         f"{(J * np_ * np_ * 20) / 1e6:.0f} MB > 129 MB L2",
                   "plan": plan},
        "roofline": {"bound": "hbm", "kernel": agent_kernel_name(plan), "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": stored_traffic(),
                     "peak_kind": f"{peak_kind} (copy bandwidth)",
                     "algorithmic_bytes_per_launch": bytes_launch,
                     "avg_launch_ms": agent_avg_ms},
        "kernels": {"agent_avg_ms": agent_avg_ms, "consensus_avg_ms": cons_avg_ms,
                    "iteration_bytes": it_bytes,
                    "iteration_GBps": it_bytes / (ms / args.steps / 1e3) / 1e9},
        "residual": {"r_fp": r_fp, "r_data": r_data},
        "gpu_launches": 2 * args.steps,
        "clocks": clocks.summary(),
        "e2e": {"value": weak_scaling_value(world, J * args.steps, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                "note": "one whole job through the C ABI from pinned host memory: create + K "
                        "iterations + residual + image readback; bytes amortised over K"},
    }
    if world == 1 and not args.no_cpu_baseline:
        rate, m, dt = oracle_rate(w, seconds=args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"one Algorithm 1 iteration (FP64 numpy, one thread) over "
                                          f"the first {m} of {J} windows, {dt:.1f} s"}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------- serving
def serving_jobs(n_jobs: int, pool_size: int, seed: int = 7):
    """Seeded job stream for the serving workload: object side in {256, 512,
    768, 1024}, probe 64 or 128 (sigma Np/4), raster step U{8..24} px with
    +-2 px jitter, Poisson peak log-uniform in [1e3, 1e6], 50-150
    iterations, FP16 amplitudes with per-pattern scales.  The measurements
    of `pool_size` distinct problems are simulated once and shared by the
    jobs (each job draws its problem, iteration count and alpha)."""
    from paper_2111_14240_gb300 import datagen
    rng = np.random.Generator(np.random.PCG64(seed))
    pool = []
    for k in range(pool_size):
        side = int(rng.choice([256, 512, 768, 1024]))
        n_p = int(rng.choice([64, 128]))
        step = int(rng.integers(8, 25))
        n_scan = (side - n_p) // step + 1
        peak = float(10 ** rng.uniform(3, 6))
        cfg = dict(n_obj=side, n_p=n_p, probe_sigma=n_p / 4, n_scan=n_scan, step=step, jitter=2,
                   peak=peak, name=f"serve{k}")
        w = datagen.make_workload(cfg, seed=1000 + k)
        codes, scales = datagen.quantize_amplitudes_f16(w.y)
        pool.append(dict(w=w, probe=w.probe.astype(np.complex64), codes=codes, scales=scales,
                         y32=w.y.astype(np.float32)))
    jobs = []
    for i in range(n_jobs):
        jobs.append(dict(p=int(rng.integers(0, pool_size)), iters=int(rng.integers(50, 151)),
                         alpha=float(rng.uniform(0.3, 1.0)), u=float(rng.random())))
    return pool, jobs


def run_serve(args):
    import torch
    from paper_2111_14240_gb300 import pmace as pm
    torch.cuda.set_device(0)
    pool, jobs = serving_jobs(args.serve_jobs, args.serve_pool)
    updates = [pool[j["p"]]["w"].J * j["iters"] for j in jobs]
    # plain FP32 single-job path: each job's service time, one at a time
    service = []
    for j in jobs:
        d = pool[j["p"]]
        w = d["w"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = pm.pmace_create(w.x.shape[0], w.x.shape[1], w.np_, w.J, KAPPA,
                            np.ascontiguousarray(d["probe"]).view(np.float32), w.offsets, d["y32"],
                            pm.PMACE_AMP_F32, inputs_on_device=False)
        pm.pmace_iterate(h, j["iters"], j["alpha"], RHO)
        img = np.empty(w.x.shape, np.complex64)
        pm.pmace_get_image(h, img)
        pm.pmace_destroy(h)
        service.append(time.perf_counter() - t0)
    total_service = sum(service)
    rate = args.serve_load * len(jobs) / total_service          # arrivals per second
    gaps = [-math.log(1.0 - j["u"]) / rate for j in jobs]
    arrivals = np.cumsum(gaps)
    # FIFO one-at-a-time latencies for the same arrivals
    t = 0.0
    lat_single = []
    for a, s in zip(arrivals, service):
        t = max(t, a) + s
        lat_single.append(t - a)
    makespan_single = t
    # serving run in real time
    srv = pm.Server(fill_pixels=args.serve_fill)
    ids = []
    t_start = time.perf_counter()
    for j, a in zip(jobs, arrivals):
        delay = t_start + a - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        d = pool[j["p"]]
        w = d["w"]
        ids.append(srv.submit(d["probe"], w.offsets, d["codes"], w.x.shape, j["iters"], j["alpha"], RHO,
                              amp_format=pm.PMACE_AMP_F16_SCALED, scales=d["scales"]))
    lat = []
    last = 0.0
    for jid in ids:
        res, _ = srv.wait(jid)
        assert res["status"] == 0, res
        lat.append((res["finish_ms"] - res["submit_ms"]) / 1e3)
        last = max(last, res["finish_ms"])
        srv.release(jid)
    makespan = time.perf_counter() - t_start
    srv.close()
    tot = float(sum(updates))
    line = {
        "metric": "PMACE serving job latency p50/p99 + patch-updates/s", "unit": "s",
        "value": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
        "higher_is_better": False, "n_gpus": 1, "jobs": len(jobs), "data": "synthetic",
        "throughput": tot / makespan, "throughput_unit": "patch-updates/s",
        "load": args.serve_load, "arrival_rate_per_s": rate, "fill_pixels": args.serve_fill,
        "single_job_fp32": {"p50": float(np.percentile(lat_single, 50)),
                            "p99": float(np.percentile(lat_single, 99)),
                            "throughput": tot / makespan_single,
                            "sum_service_s": total_service},
        "config": {"workload": "serving: seeded job stream, Poisson arrivals at the given fraction of the "
                               "single-job path's capacity; object side {256,512,768,1024}, probe 64/128, "
                               "step 8-24 px +-2, peak 1e3-1e6, 50-150 iterations, FP16 amplitudes; "
                               f"{args.serve_pool} distinct problems shared by {len(jobs)} jobs"},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_convergence(args):
    """Reconstruction error against iteration on the 324-window workload for
    the alpha / kappa grid whose FP64 oracle curves are stored under
    tests/golden (read as data; the oracle is not run here).  NRMSE as in
    Section IV: global phase aligned, over the pixels some window covers."""
    import glob
    import torch

    from paper_2111_14240_gb300 import build, datagen
    from paper_2111_14240_gb300 import pmace as pm
    build.build()
    curves = []
    golden = os.path.join(ROOT, "tests", "golden")
    # the oracle at the bench's parameters under rounding-sized perturbations
    # (inputs, and inputs plus stored state, in single precision): how far its
    # own error curve moves when nothing but rounding changes
    spread = {}
    for path in sorted(glob.glob(os.path.join(golden, "nrmse_p256_spread_*.json"))):
        with open(path) as f:
            g = json.load(f)
        spread[g["perturbation"]] = [pt["nrmse"] for pt in g["points"]]
    for path in sorted(glob.glob(os.path.join(golden, "nrmse_p256*.json"))):
        if "_spread_" in path:
            continue
        with open(path) as f:
            g = json.load(f)
        w = datagen.make_workload(g["workload"], seed=g["seed"])
        mask = np.zeros(w.x.shape, bool)
        for r, c in w.offsets:
            mask[r:r + w.np_, c:c + w.np_] = True
        x_true = w.x[mask]
        rec = pm.Reconstruction(w.probe.astype(np.complex64), w.offsets, w.y.astype(np.float32), w.x.shape,
                                kappa=g["kappa"])
        pts, done, t_iter = [], 0, 0.0
        for pt in g["points"]:
            n = pt["iteration"] - done
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rec.iterate(n, g["alpha"], g["rho"])
            torch.cuda.synchronize()
            t_iter += time.perf_counter() - t0
            done = pt["iteration"]
            xh = rec.image().cpu().numpy().astype(np.complex128)[mask]
            theta = np.angle(np.vdot(x_true, xh))
            e = float(np.linalg.norm(xh - np.exp(1j * theta) * x_true) / np.linalg.norm(x_true))
            pts.append({"iteration": done, "nrmse_gpu": e, "nrmse_oracle": pt["nrmse"]})
        r_fp, r_data = rec.residual()
        rec.close()
        c = {"alpha": g["alpha"], "kappa": g["kappa"], "rho": g["rho"], "points": pts,
             "final_rel_diff": abs(pts[-1]["nrmse_gpu"] - pts[-1]["nrmse_oracle"]) / pts[-1]["nrmse_oracle"],
             "ms_per_iteration": 1e3 * t_iter / done, "r_fp": r_fp, "r_data": r_data}
        if os.path.basename(path) == "nrmse_p256.json" and spread:
            c["oracle_rounding_runs"] = {k: v for k, v in spread.items()}
            c["oracle_rounding_spread_final"] = max(abs(v[-1] - pts[-1]["nrmse_oracle"]) / pts[-1]["nrmse_oracle"]
                                                    for v in spread.values())
        curves.append(c)
    best = min(curves, key=lambda c: c["points"][-1]["nrmse_gpu"])
    print(json.dumps({"metric": "PMACE reconstruction NRMSE vs iteration (alpha / kappa sweep)",
                      "unit": "NRMSE", "value": best["points"][-1]["nrmse_gpu"], "higher_is_better": False,
                      "n_gpus": 1, "data": "synthetic", "dtype": "f32",
                      "config": {"workload": WORKLOAD, "start": "energy-matched constant",
                                 "best": {"alpha": best["alpha"], "kappa": best["kappa"]}},
                      "curves": curves}))
    return 0


def run_simulate(args):
    """Throughput of the GPU data simulator (pmace_simulate) on the p256
    geometry, noisy (peak 1e5), inputs and output resident on the device."""
    import torch

    from paper_2111_14240_gb300 import build, datagen
    from paper_2111_14240_gb300 import pmace as pm
    build.build()
    w = datagen.make_workload("p256", seed=1)
    x = torch.from_numpy(w.x.astype(np.complex64)).cuda()
    d = torch.from_numpy(w.probe.astype(np.complex64)).cuda()
    out = torch.empty((w.J, w.np_, w.np_), dtype=torch.float32, device="cuda")
    dims = pm.pmace_dims(w.x.shape[0], w.x.shape[1], w.np_, w.J, 1.0)
    offs = np.ascontiguousarray(w.offsets, dtype=np.int32)

    def once():
        pm._check(pm._lib.pmace_simulate(pm.ctypes.byref(dims), pm._ptr(d), pm._ptr(offs), pm._ptr(x), 1e5, 7,
                                         pm._ptr(out), 1, pm._stream(None)), None)

    for _ in range(max(args.warmup, 3)):
        once()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        once()
    torch.cuda.synchronize()
    s = (time.perf_counter() - t0) / args.steps
    moved = w.J * w.np_ ** 2 * (8 + 8 + 8 + 4 + 4 + 4)   # rows write S, columns read S, intensity w/r, y
    print(json.dumps({"metric": "PMACE simulated patterns/s", "value": w.J / s, "unit": "patterns/s",
                      "higher_is_better": True, "n_gpus": 1, "steps": args.steps, "ms_per_step": s * 1e3,
                      "data": "synthetic", "dtype": "f32 (FFT), f64 (noise)",
                      "config": {"workload": WORKLOAD, "peak": 1e5, "timed": "whole pmace_simulate call "
                                 "(scratch allocation, three kernels, synchronisation); inputs on the device"},
                      "bytes_per_step": moved, "GBps": moved / s / 1e9}))
    return 0


def _nrmse(x_hat, x, mask):
    """Section IV NRMSE with the global phase chosen to minimise it, over `mask`."""
    a, b = x_hat[mask].astype(np.complex128), x[mask]
    theta = np.angle(np.vdot(b, a))
    return float(np.linalg.norm(a - np.exp(1j * theta) * b) / np.linalg.norm(b))


def precision_case(cfg, peak, iters, seed=1, stream=None):
    """One workload of the precision comparison: measurements made by the GPU
    simulator, then `iters` iterations on FP32 amplitudes and on FP16 codes
    with per-pattern scales.  Returns (nrmse32, nrmse16, ms32, ms16, J)."""
    import torch

    from paper_2111_14240_gb300 import datagen
    from paper_2111_14240_gb300 import pmace as pm
    rng = np.random.Generator(np.random.PCG64(seed))
    x = datagen.make_object(rng, cfg["n_obj"], cfg["n_obj"])
    probe = datagen.make_probe(rng, cfg["n_p"], cfg["probe_sigma"])
    offs = datagen.make_offsets(rng, cfg["n_obj"], cfg["n_p"], cfg["n_scan"], cfg["step"], cfg["jitter"])
    y = pm.simulate(x, probe, offs, peak=peak, seed=seed)
    mask = np.zeros(x.shape, bool)
    for r, c in offs:
        mask[r:r + cfg["n_p"], c:c + cfg["n_p"]] = True
    codes, scales = datagen.quantize_amplitudes_f16(y.astype(np.float64))
    out = []
    for f16 in (False, True):
        if f16:
            rec = pm.Reconstruction(probe.astype(np.complex64), offs, torch.from_numpy(codes).cuda(), x.shape,
                                    amp_format=pm.PMACE_AMP_F16_SCALED, scales=torch.from_numpy(scales).cuda())
        else:
            rec = pm.Reconstruction(probe.astype(np.complex64), offs, y, x.shape)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rec.iterate(iters, ALPHA, RHO)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / iters
        out.append((_nrmse(rec.image().cpu().numpy(), x, mask), ms))
        rec.close()
        torch.cuda.empty_cache()
    return out[0][0], out[1][0], out[0][1], out[1][1], len(offs)


def run_precision(args):
    """FP16 amplitudes (per-pattern scale) against FP32 on the 2048^2 /
    128 x 128 / 14641-window workload at Poisson peaks 1e4 and 1e6, 200
    iterations each, measurements from the GPU simulator."""
    from paper_2111_14240_gb300 import build, datagen
    build.build()
    cfg = datagen.CONFIGS["p128"]
    rows = []
    for peak in (1e4, 1e6):
        e32, e16, ms32, ms16, J = precision_case(cfg, peak, 200)
        rows.append({"peak": peak, "nrmse_fp32": e32, "nrmse_fp16": e16, "rel_diff": abs(e16 - e32) / e32,
                     "ms_per_iteration_fp32": ms32, "ms_per_iteration_fp16": ms16,
                     "patch_updates_per_s_fp32": J / ms32 * 1e3, "patch_updates_per_s_fp16": J / ms16 * 1e3})
    print(json.dumps({"metric": "PMACE FP16-amplitude path against FP32: NRMSE and patch-updates/s",
                      "unit": "NRMSE relative difference", "value": max(r["rel_diff"] for r in rows),
                      "higher_is_better": False, "n_gpus": 1, "data": "synthetic (GPU simulator)",
                      "config": {"workload": "2048x2048 object, 128x128 probe (sigma 32 px), 121x121 raster step "
                                             "16 px +-2 = 14641 windows, 200 iterations, alpha 0.5, rho 0.5"},
                      "runs": rows}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=0.0,
                    help="reference arm: seconds of oracle work per step (0: sized for a few minutes)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve", action="store_true", help="run the serving workload instead")
    ap.add_argument("--serve-jobs", type=int, default=256)
    ap.add_argument("--serve-pool", type=int, default=16)
    ap.add_argument("--serve-load", type=float, default=0.8)
    ap.add_argument("--serve-fill", type=int, default=0, help="server fill target in pixels (0: default)")
    ap.add_argument("--convergence", action="store_true",
                    help="reconstruction error against iteration over the stored alpha / kappa grid")
    ap.add_argument("--simulate", action="store_true", help="time the GPU data simulator instead")
    ap.add_argument("--precision", action="store_true",
                    help="FP16 against FP32 amplitudes on the 14641-window workload")
    args = ap.parse_args()
    if args.serve:
        return run_serve(args)
    if args.convergence:
        return run_convergence(args)
    if args.simulate:
        return run_simulate(args)
    if args.precision:
        return run_precision(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
