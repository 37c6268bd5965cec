"""Benchmark of the PMACE hot path on GB300: patch-updates/s.

A step is one PMACE iteration (Algorithm 1) over every window of the
workload: the fused agent sweep (steps S0-S5) and the consensus gather (S6),
two kernel launches.  The default workload is the largest single scan that
fits one GPU: an 8192 x 8192 complex object, a 128 x 128 probe (Gaussian,
sigma 32 px, random quadratic phase) and a 253 x 253 raster with a step of
32 px and +-3 px jitter (64009 windows), FP16 amplitudes with a per-pattern
FP32 scale at Poisson peak 1e5.  The object, probe and scan come from the
seeded generator (a synthetic stand-in for the paper's LANL image and
probe, which are not available); the amplitudes are made on the GPU by the
library's simulator, outside the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload large|p128|p256|small]

One JSON line is printed by rank 0.  Under torchrun every rank runs an
independent replica of the job on its own GPU (no data-path collective;
"scaling": "weak"); the time is the maximum over ranks.  `--impl reference`
times the FP64 CPU oracle instead (rank 0 only), on a bounded sample of the
same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import functools
import hashlib
import json
import math
import os
import platform
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

# name -> (generator configuration, FP16 amplitudes, photon peak, description)
WORKLOADS = {
    "large": ("large", True, 1e5,
              "largest single scan: object 8192x8192 complex64, probe 128x128 (Gaussian sigma 32 px, random "
              "quadratic phase), 253x253 raster step 32 px +-3 px jitter = 64009 windows, FP16 amplitudes with "
              "per-pattern FP32 scale, Poisson peak 1e5, alpha 0.5, rho 0.5, kappa 1.25"),
    "p128": ("p128", True, 1e4,
             "precision path: object 2048x2048, probe 128x128 (sigma 32 px), 121x121 raster step 16 px +-2 px = "
             "14641 windows, FP16 amplitudes with per-pattern FP32 scale, Poisson peak 1e4, alpha 0.5, rho 0.5, "
             "kappa 1.25"),
    "p128_f32": ("p128", False, 1e4,
                 "precision path with FP32 amplitudes: object 2048x2048, probe 128x128, 14641 windows, Poisson "
                 "peak 1e4"),
    "p256": ("p256", False, 1e5,
             "object 600x600 complex64, probe 256x256 (Gaussian sigma 48 px, random quadratic phase), 18x18 "
             "raster step 20 px +-2 px = 324 windows, FP32 amplitudes, Poisson peak 1e5"),
    "small": ("small", False, 1e5,
              "object 128x128, probe 32x32 (sigma 8 px), 13x13 raster step 8 px +-1 px = 169 windows, FP32 "
              "amplitudes, Poisson peak 1e5"),
}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "agent_traffic.json")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2111_14240_gb300", "csrc", f)
                  for f in ("agent.cuh", "agent_xpose.cuh", "agent_pair.cuh", "cache_hints.cuh", "tmem.cuh",
                            "fft_smem.cuh", "pmace_internal.h")]


def kernel_hash() -> str:
    """Hash of the agent kernels' source code with comments and blank space
    removed, so that a comment edit does not orphan the stored counters."""
    import re
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        if not os.path.exists(p):
            continue
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


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """SM clocks and clock-event (throttle) reasons sampled every `period`
    seconds during the timed region, by read-only NVML queries through
    ctypes (nvidia-smi at 100 ms if NVML cannot be loaded)."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, index: int, period: float = 0.01):
        self.index, self.period = index, period
        self.samples = []          # (sm_mhz, max_mhz, reasons bitmask)
        self._stop = threading.Event()
        self._nvml = self._handle = None
        self._proc = None
        self.source = "none"

    def _open_nvml(self):
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return False
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(h)) != 0:
                return False
            self._nvml, self._handle = lib, h
            self._reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
            return True
        except (OSError, AttributeError):
            return False

    def _sample_nvml(self):
        sm, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        lib, h = self._nvml, self._handle
        while not self._stop.is_set():
            if (lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(sm)) == 0
                    and lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0
                    and self._reasons_fn(h, ctypes.byref(rs)) == 0):
                self.samples.append((float(sm.value), float(mx.value), int(rs.value)))
            time.sleep(self.period)

    def _read_smi(self):
        names = [0x8, 0x40, 0x20, 0x4]
        for line in self._proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 6:
                continue
            try:
                bits = sum(b for b, v in zip(names, parts[2:6]) if v.lower().startswith("active"))
                self.samples.append((float(parts[0]), float(parts[1]), bits))
            except ValueError:
                continue

    def __enter__(self):
        if self._open_nvml():
            self.source = f"nvml every {self.period * 1e3:.0f} ms"
            self._thread = threading.Thread(target=self._sample_nvml, daemon=True)
            self._thread.start()
        else:
            try:
                self._proc = subprocess.Popen(
                    ["nvidia-smi", "-i", str(self.index),
                     "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
                     "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                     "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "100"],
                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
                self.source = "nvidia-smi every 100 ms"
                self._thread = threading.Thread(target=self._read_smi, daemon=True)
                self._thread.start()
            except OSError:
                self._proc = None
        return self

    def __exit__(self, *exc):
        self._stop.set()
        if self._proc is not None:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self._proc.kill()
        if getattr(self, "_thread", None) is not None:
            self._thread.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0,
                    "source": self.source}
        bits = 0
        for _, _, b in self.samples:
            bits |= b
        return {"sm_mhz": statistics.median(s for s, _, _ in self.samples),
                "sm_max_mhz": max(m for _, m, _ in self.samples),
                "reasons": sorted(n for b, n in self.REASONS.items() if bits & b),
                "samples": len(self.samples), "source": self.source}


# ------------------------------------------------------------------ ranks
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
    """The agent sweep kernel a plan launches."""
    return {0: "agent_kernel", 1: "agent_xpose_kernel", 2: "agent_pair_kernel"}.get(plan.get("exchange"), "?")


def stored_traffic(workload: str, J: int):
    """DRAM bytes per launch of the agent sweep from the stored ncu counters,
    when they were taken on the current kernel source: per window of the
    captured case times the windows of one launch (the traffic grows with
    the windows processed), else None."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    with open(TRAFFIC_FILE) as f:
        d = json.load(f)
    e = d.get(workload)
    if not e or e.get("kernel_hash") != kernel_hash():
        return None
    return float(e["bytes_per_window"]) * J


def host_info():
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
        for key in ("model name", "Model", "CPU part"):
            for line in info.splitlines():
                if line.startswith(key):
                    model = line.split(":", 1)[1].strip()
                    break
            if model:
                break
    except OSError:
        pass
    # Arm reports a part number, not a name
    parts = {"0xd4f": "Arm Neoverse V2 (part 0xd4f)", "0xd40": "Arm Neoverse V1 (part 0xd40)",
             "0xd0c": "Arm Neoverse N1 (part 0xd0c)", "0xd8e": "Arm Neoverse N3 (part 0xd8e)"}
    model = parts.get(model, model)
    return {"cpu_count": os.cpu_count(), "cpu_model": model or platform.processor() or platform.machine(),
            "machine": platform.machine()}


# ------------------------------------------------------------------ inputs
# --scan n: an n x n sub-raster of the headline workload's scan (the same
# object, probe and step), for profiling captures of a few GB
SCAN_OVERRIDE = {}


@functools.lru_cache(maxsize=2)
def scan_geometry(name: str, seed: int = 1):
    """Object, probe and scan offsets of a workload, drawn in the generator's
    order (the amplitudes are made separately)."""
    from paper_2111_14240_gb300 import datagen
    c = datagen.CONFIGS[WORKLOADS[name][0]]
    rng = np.random.Generator(np.random.PCG64(seed))
    x = datagen.make_object(rng, c["n_obj"], c["n_obj"])
    probe = datagen.make_probe(rng, c["n_p"], c["probe_sigma"])
    offs = datagen.make_offsets(rng, c["n_obj"], c["n_p"], SCAN_OVERRIDE.get(name, c["n_scan"]), c["step"],
                                c["jitter"])
    return x, probe, offs


def device_inputs(name: str, seed: int = 1):
    """A workload's inputs with the amplitudes resident on the GPU: made by
    the library's simulator (Section II forward model, Section IV photon
    scaling) and, for the FP16 path, stored as float16 codes y_j / s_j with
    s_j = max y_j.  Returns (x, probe complex64, offsets, amps, scales)."""
    import torch

    from paper_2111_14240_gb300 import pmace as pm
    cfg, f16, peak, _ = WORKLOADS[name]
    x, probe, offs = scan_geometry(name, seed)
    n1, n2 = x.shape
    np_ = probe.shape[0]
    J = offs.shape[0]
    probe32 = np.ascontiguousarray(probe.astype(np.complex64))
    xd = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
    dd = torch.from_numpy(probe32).cuda()
    y = torch.empty((J, np_, np_), dtype=torch.float32, device="cuda")
    dims = pm.pmace_dims(n1, n2, np_, J, 1.0)
    o32 = np.ascontiguousarray(offs, dtype=np.int32)
    pm._check(pm._lib.pmace_simulate(ctypes.byref(dims), pm._ptr(dd), pm._ptr(o32), pm._ptr(xd), float(peak),
                                     7 + seed, pm._ptr(y), 1, pm._stream(None)), None)
    del xd, dd
    if not f16:
        return x, probe32, o32, y, None
    s = y.reshape(J, -1).amax(dim=1)
    s = torch.where(s > 0, s, torch.ones_like(s)).contiguous()
    codes = (y / s[:, None, None]).to(torch.float16).contiguous()
    del y
    torch.cuda.empty_cache()
    return x, probe32, o32, codes, s


def host_inputs(name: str, m: int | None = None, seed: int = 1):
    """CPU-only inputs of the first m windows of a workload for the FP64
    oracle: the generator's object, probe and scan, measurements of those
    windows by the generator's float64 forward model with Poisson noise, and
    for the FP16 path the dequantised codes (code * scale, exact in FP64).
    The image is cut to the rows those windows cover.  Returns (y, probe,
    offsets, shape)."""
    from paper_2111_14240_gb300 import datagen
    _, f16, peak, _ = WORKLOADS[name]
    x, probe, offs = scan_geometry(name, seed)
    offs = offs if m is None else offs[:m]
    np_ = probe.shape[0]
    rows = int(offs[:, 0].max()) + np_
    x = x[:rows]
    y = datagen.simulate(np.random.Generator(np.random.PCG64(seed + 100)), x, probe, offs, peak)
    if f16:
        codes, scales = datagen.quantize_amplitudes_f16(y)
        y = datagen.dequantize_f16(codes, scales)
    return y, probe, np.ascontiguousarray(offs), x.shape


# ------------------------------------------------------------------ oracle
def oracle_baseline(name: str, seconds: float, max_windows: int, n_iter: int = 2):
    """The FP64 oracle on the host cores, on the first m windows of the
    workload, m sized so that n_iter iterations take about `seconds`:
    (a) the literal single-thread Algorithm 1 (oracle/pmace_oracle.py),
    (b) the batched variant with scipy.fft on every core
    (oracle/pmace_batched.py).  Returns both as cpu_baseline records."""
    from oracle import pmace_batched
    from oracle import pmace_oracle as orc
    J_full = None
    out = {}
    y, probe, offs, shape = host_inputs(name, m=min(16, max_windows))
    t0 = time.perf_counter()
    orc.pmace(y, probe, offs, shape, alpha=ALPHA, rho=RHO, kappa=KAPPA, n_iter=1)
    per = (time.perf_counter() - t0) / len(offs)
    m = max(16, min(max_windows, int(seconds / n_iter / max(per, 1e-6))))
    y, probe, offs, shape = host_inputs(name, m=m)
    from paper_2111_14240_gb300 import datagen
    c = datagen.CONFIGS[WORKLOADS[name][0]]
    J_full = c["n_scan"] ** 2
    cores = os.cpu_count() or 1
    for kind, fn, threads in (("literal", orc.pmace, 1), ("batched", pmace_batched.pmace, cores)):
        kw = dict(alpha=ALPHA, rho=RHO, kappa=KAPPA, n_iter=n_iter)
        if kind == "batched":
            kw["workers"] = cores
        t0 = time.perf_counter()
        fn(y, probe, offs, shape, **kw)
        dt = time.perf_counter() - t0
        rate = len(offs) * n_iter / dt
        what = ("Algorithm 1 as written (oracle/pmace_oracle.py: FP64 numpy, one thread)" if kind == "literal"
                else f"Algorithm 1 with the agents of the stack taken by scipy.fft on {cores} threads "
                     f"(oracle/pmace_batched.py, FP64)")
        out[kind] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                     "sample": f"{what}: {n_iter} iterations over the first {len(offs)} of {J_full} windows "
                               f"({dt:.1f} s), the rate extrapolated to the whole scan"}
    return out


def run_reference(args):
    dist, world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    from oracle import pmace_oracle as orc
    name = args.workload
    budget = 150.0
    per_step = max(0.2, min(6.0, budget / max(1, args.steps + args.warmup)))
    if args.ref_seconds > 0:
        per_step = args.ref_seconds
    y, probe, offs, shape = host_inputs(name, m=8)
    t0 = time.perf_counter()
    orc.pmace(y, probe, offs, shape, alpha=ALPHA, rho=RHO, kappa=KAPPA, n_iter=1)
    per = (time.perf_counter() - t0) / len(offs)
    m = max(1, int(per_step / per))
    y, probe, offs, shape = host_inputs(name, m=m)
    m = len(offs)
    v = None
    for _ in range(args.warmup):
        v = orc.pmace(y, probe, offs, shape, alpha=ALPHA, rho=RHO, kappa=KAPPA, n_iter=1, v0=v)["v"]
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v = orc.pmace(y, probe, offs, shape, alpha=ALPHA, rho=RHO, kappa=KAPPA, n_iter=1, v0=v)["v"]
    dt = time.perf_counter() - t0
    val = m * args.steps / dt
    from paper_2111_14240_gb300 import datagen
    J = datagen.CONFIGS[WORKLOADS[name][0]]["n_scan"] ** 2
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOADS[name][3]},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"Algorithm 1 (FP64 numpy, single thread) over the first {m} of "
                                   f"{J} windows per step, the rate extrapolated to the whole scan; each "
                                   f"step one iteration"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "host": host_info(),
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ ours
def time_job(rec, steps: int, warmup: int, stream, clocks_index=None, dist=None):
    """Warm up, then time `steps` iterations with CUDA events on the job's
    stream (barrier + synchronize on both sides); per-kernel times from the
    library's own event pairs.  Returns (ms, kernel times, clocks)."""
    import torch

    from paper_2111_14240_gb300 import pmace as pm
    rec.iterate(warmup, ALPHA, RHO)
    torch.cuda.synchronize()
    pm.pmace_set_profiling(rec.h, True)
    pm.pmace_kernel_times(rec.h, reset=True)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(clocks_index) if clocks_index is not None else None
    if sampler:
        sampler.__enter__()
    try:
        start.record(stream)
        rec.iterate(steps, ALPHA, RHO)
        stop.record(stream)
        torch.cuda.synchronize()
    finally:
        if sampler:
            sampler.__exit__(None, None, None)
    if dist:
        dist.barrier()
    ms = start.elapsed_time(stop)
    kt = pm.pmace_kernel_times(rec.h, reset=True)
    pm.pmace_set_profiling(rec.h, False)
    return ms, kt, (sampler.summary() if sampler else None)


def roofline_of(kt, J, np_, amp_bytes, workload):
    peak, peak_kind = measured_peaks()
    agent_avg_ms = kt["agent_ms"] / max(1, kt["agent_launches"])
    bytes_launch = J * agent_bytes_per_patch(np_, amp_bytes)
    achieved = bytes_launch / (agent_avg_ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": stored_traffic(workload, J), "peak_kind": f"{peak_kind} copy bandwidth (burst)",
            "algorithmic_bytes_per_launch": bytes_launch,
            "algorithmic_bytes_per_window": agent_bytes_per_patch(np_, amp_bytes), "avg_launch_ms": agent_avg_ms}


def agent_flops_per_window(np_: int) -> int:
    """Nominal FP32 operations of one window's agent update: 10 P log2 P for
    the forward and inverse 2-D transforms and about 45 P for the probe
    products, the magnitude replacement and the update (P = Np^2)."""
    P = np_ * np_
    return int(10 * P * math.log2(P) + 45 * P)


def fp32_peak_tflops() -> float:
    """FP32 (CUDA-core) throughput of the device: a float32 matrix product
    of 8192^3 with TF32 off, best of 5 (CUDA events)."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        n = 8192
        g = torch.Generator(device="cuda").manual_seed(0)
        a = torch.randn(n, n, device="cuda", generator=g)
        b = torch.randn(n, n, device="cuda", generator=g)
        for _ in range(2):
            c = a @ b
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = float("inf")
        for _ in range(5):
            e0.record()
            c = a @ b
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        del a, b, c
        torch.cuda.empty_cache()
        return 2.0 * n ** 3 / (best / 1e3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def extra_workload(name: str, steps: int, warmup: int, stream):
    """Throughput and agent roofline of another workload (device-resident
    inputs), for the record beside the headline."""
    import torch

    from paper_2111_14240_gb300 import datagen
    from paper_2111_14240_gb300 import pmace as pm
    cfg, f16, _, desc = WORKLOADS[name]
    if name == "p256":
        w = datagen.make_workload("p256", seed=1)
        x_shape, probe32, offs = w.x.shape, w.probe.astype(np.complex64), w.offsets
        amps, scales = torch.from_numpy(w.y.astype(np.float32)).cuda(), None
    else:
        x, probe32, offs, amps, scales = device_inputs(name)
        x_shape = x.shape
    J, np_ = len(offs), probe32.shape[0]
    rec = pm.Reconstruction(probe32, offs, amps, x_shape, kappa=KAPPA, stream=stream,
                            amp_format=pm.PMACE_AMP_F16_SCALED if f16 else pm.PMACE_AMP_F32, scales=scales)
    del amps
    ms, kt, _ = time_job(rec, steps, warmup, stream)
    plan = rec.plan()
    rec.close()
    torch.cuda.empty_cache()
    n1, n2 = x_shape
    amp_b = 2 if f16 else 4
    it_ms = ms / steps
    return {"workload": desc, "value": J * steps / (ms / 1e3), "unit": UNIT, "steps": steps,
            "ms_per_step": it_ms, "agent_avg_ms": kt["agent_ms"] / max(1, kt["agent_launches"]),
            "consensus_avg_ms": kt["consensus_ms"] / max(1, kt["consensus_launches"]),
            "roofline": roofline_of(kt, J, np_, amp_b, name),
            "iteration_frac_of_hbm": iteration_bytes(np_, J, n1, n2, amp_b) / (it_ms / 1e3) / 1e9
            / measured_peaks()[0], "plan": plan}


def run_ours(args):
    import torch
    dist, world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    from paper_2111_14240_gb300 import pmace as pm

    name = args.workload
    cfg, f16, peak, desc = WORKLOADS[name]
    stream = torch.cuda.current_stream()
    x, probe32, offs, amps, scales = device_inputs(name)
    n1, n2 = x.shape
    J, np_ = len(offs), probe32.shape[0]
    amp_b = 2 if f16 else 4
    fmt = pm.PMACE_AMP_F16_SCALED if f16 else pm.PMACE_AMP_F32

    # host copies for the end-to-end run (pinned)
    amps_pin = amps.cpu().pin_memory()
    scales_pin = scales.cpu().pin_memory() if scales is not None else None
    p_pin = torch.view_as_real(torch.from_numpy(probe32)).contiguous().pin_memory()

    rec = pm.Reconstruction(probe32, offs, amps, (n1, n2), kappa=KAPPA, stream=stream, amp_format=fmt,
                            scales=scales)
    del amps
    plan = rec.plan()
    ms, kt, clocks = time_job(rec, args.steps, args.warmup, stream, clocks_index=local, dist=dist)
    r_fp, r_data = rec.residual()
    rec.close()
    torch.cuda.empty_cache()

    # end to end through the C ABI from pinned host buffers: create (H2D of
    # probe, offsets, amplitudes and scales), K iterations, residual and
    # image (D2H)
    img_pin = torch.empty((n1, n2, 2), dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    h = pm.pmace_create(n1, n2, np_, J, KAPPA, p_pin, offs, amps_pin, fmt, scales=scales_pin,
                        inputs_on_device=False, stream=stream)
    pm.pmace_iterate(h, args.steps, ALPHA, RHO, stream=stream)
    pm.pmace_residual(h, stream=stream)
    pm.pmace_get_image(h, img_pin, stream=stream)
    e2e_s = time.perf_counter() - t0
    pm.pmace_destroy(h)
    h2d = amps_pin.numel() * amps_pin.element_size() + probe32.nbytes + offs.nbytes + (
        scales_pin.numel() * 4 if scales_pin is not None else 0)
    d2h = img_pin.numel() * 4 + 16
    del amps_pin, scales_pin, img_pin
    torch.cuda.empty_cache()

    ms, e2e_s = max_over_ranks(dist, [ms, e2e_s])
    if rank != 0:
        return 0

    value = weak_scaling_value(world, J * args.steps, ms / 1e3)
    cons_avg_ms = kt["consensus_ms"] / max(1, kt["consensus_launches"])
    it_bytes = iteration_bytes(np_, J, n1, n2, amp_b)
    roof = roofline_of(kt, J, np_, amp_b, name)
    roof["kernel"] = agent_kernel_name(plan)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP16 amplitudes)" if f16 else "f32",
        "data": "synthetic (seeded generator; amplitudes by the GPU simulator)",
        "config": {"workload": desc if not args.scan else f"{args.scan}x{args.scan} sub-raster of: {desc}",
                   "windows": J, "probe": np_, "image": [n1, n2],
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "no flush: per-step working set (q, u, y) is "
                         f"{(J * np_ * np_ * (16 + amp_b)) / 1e9:.2f} GB > 129 MB L2",
                   "plan": plan},
        "roofline": roof,
        "kernels": {"agent_avg_ms": roof["avg_launch_ms"], "consensus_avg_ms": cons_avg_ms,
                    "iteration_bytes": it_bytes,
                    "iteration_GBps": it_bytes / (ms / args.steps / 1e3) / 1e9,
                    "iteration_frac_of_hbm": it_bytes / (ms / args.steps / 1e3) / 1e9 / roof["peak"]},
        "residual": {"r_fp": r_fp, "r_data": r_data},
        "gpu_launches": 2 * args.steps,
        "clocks": clocks,
        "e2e": {"value": weak_scaling_value(world, J * args.steps, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                "note": "one whole job through the C ABI from pinned host memory: create + K "
                        "iterations + residual + image readback; bytes amortised over K"},
        "host": host_info(),
    }
    if world == 1:
        fp = fp32_peak_tflops()
        fl = agent_flops_per_window(np_)
        ach = J * fl / (roof["avg_launch_ms"] / 1e3) / 1e12
        line["kernels"]["agent_fp32"] = {
            "flops_per_window": fl, "achieved_tflops": ach, "peak_tflops": fp, "frac": ach / fp,
            "peak_kind": "measured float32 matrix product, TF32 off (CUDA cores), best of 5",
            "note": "nominal FFT and update operations (10 P log2 P + 45 P, P = Np^2) per launch / average launch time"}
    if world == 1 and not args.no_extra:
        line["extra"] = {}
        for other in ("p256", "p128", "p128_f32"):
            if other != name:
                line["extra"][other] = extra_workload(other, args.extra_steps, args.warmup, stream)
    if world == 1 and not args.no_serving:
        line["serving"] = serving_record(args.serve_small_jobs, args.serve_small_pool, args.serve_load,
                                         args.serve_fill)
    if world == 1 and not args.no_cpu_baseline:
        cb = oracle_baseline(name, args.cpu_seconds, args.cpu_max_windows)
        line["cpu_baseline"] = cb["literal"]
        line["cpu_baseline_batched"] = cb["batched"]
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


def serving_record(n_jobs: int, pool_size: int, load: float, fill: int = 0):
    """The serving workload at `load` times the single-job path's capacity:
    each job's service time alone on the plain FP32 single-job path, then
    the same jobs through the continuous-batching server in real time with
    Poisson arrivals.  Returns p50 / p99 job latency of both and the
    throughput."""
    import torch
    from paper_2111_14240_gb300 import pmace as pm
    pool, jobs = serving_jobs(n_jobs, pool_size)
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
    rate = load * len(jobs) / total_service          # arrivals per second
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
    srv = pm.Server(fill_pixels=fill)
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
    for jid in ids:
        res, _ = srv.wait(jid)
        assert res["status"] == 0, res
        lat.append((res["finish_ms"] - res["submit_ms"]) / 1e3)
        srv.release(jid)
    makespan = time.perf_counter() - t_start
    srv.close()
    tot = float(sum(updates))
    return {
        "metric": "PMACE serving job latency p50/p99 + patch-updates/s", "unit": "s",
        "p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
        "jobs": len(jobs), "throughput": tot / makespan, "throughput_unit": "patch-updates/s",
        "load": load, "arrival_rate_per_s": rate, "fill_pixels": fill,
        "single_job_fp32": {"p50": float(np.percentile(lat_single, 50)),
                            "p99": float(np.percentile(lat_single, 99)),
                            "throughput": tot / makespan_single, "sum_service_s": total_service},
        "workload": "serving: seeded job stream, Poisson arrivals at the given fraction of the single-job "
                    "path's capacity; object side {256,512,768,1024}, probe 64/128, step 8-24 px +-2, peak "
                    f"1e3-1e6, 50-150 iterations, FP16 amplitudes; {pool_size} distinct problems shared by "
                    f"{len(jobs)} jobs; the single-job path runs FP32 amplitudes one job at a time (FIFO)",
    }


def run_serve(args):
    import torch
    torch.cuda.set_device(0)
    r = serving_record(args.serve_jobs, args.serve_pool, args.serve_load, args.serve_fill)
    line = dict(r, value=r["p50"], higher_is_better=False, n_gpus=1, data="synthetic",
                config={"workload": r.pop("workload")})
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
                      "config": {"workload": WORKLOADS["p256"][3], "start": "energy-matched constant",
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
                      "config": {"workload": WORKLOADS["p256"][3], "peak": 1e5, "timed": "whole pmace_simulate call "
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
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS),
                    help="the headline workload (default: the 64009-window 8192^2 scan)")
    ap.add_argument("--scan", type=int, default=0,
                    help="n x n sub-raster of the workload's scan (profiling captures; 0: the full scan)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="seconds of oracle work per CPU-baseline variant")
    ap.add_argument("--cpu-max-windows", type=int, default=4096)
    ap.add_argument("--ref-seconds", type=float, default=0.0,
                    help="reference arm: seconds of oracle work per step (0: sized for a few minutes)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the other workloads' records")
    ap.add_argument("--extra-steps", type=int, default=50)
    ap.add_argument("--no-serving", action="store_true", help="skip the compact serving record")
    ap.add_argument("--serve-small-jobs", type=int, default=32)
    ap.add_argument("--serve-small-pool", type=int, default=8)
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
    if args.scan > 0:
        SCAN_OVERRIDE[args.workload] = args.scan
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
