"""Write the FP64 oracle's reconstruction-error curves used by the GPU tests.

Runs Algorithm 1 of the oracle (and nothing else) on seeded synthetic
workloads from the energy-matched constant start and records the NRMSE of
Section IV (global phase aligned, over the pixels some window covers) of
the readout x_hat after every `every` iterations.  Usage:

    python tests/golden/make_nrmse_curves.py

writes tests/golden/nrmse_<name>[_a<alpha>_k<kappa>].json.  Deterministic:
the workloads come from seeded generators and the oracle is plain FP64 numpy.

It also writes tests/golden/nrmse_<name>_spread_<perturbation>.json: the same
oracle run at the bench's parameters with perturbations of the size of
single-precision rounding, which measure how far the oracle's own error
curve moves when nothing but rounding changes:

  in32          the probe rounded to complex64 and the amplitudes to float32
                (the inputs exactly as the GPU receives them);
  in32_state32  the same inputs, and the carried state (the stack v and the
                consensus stack z) rounded to complex64 after every
                iteration, as single-precision storage would;
  in32_fft32    the same inputs, and the oracle's two transforms (fft2o,
                ifft2o) evaluated in single precision (numpy's complex64
                FFT), everything else in FP64: the rounding of a
                single-precision FFT, which the GPU path also incurs.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "..", ".."))

from oracle import pmace_oracle as orc  # noqa: E402
from paper_2111_14240_gb300 import datagen  # noqa: E402

# (workload, seed, iterations, every, alpha, rho, kappa): the 600 x 600 /
# 256 x 256 / 324-window geometry at the bench's parameters, then a sweep of
# the noise-to-signal ratio alpha and the probe exponent kappa (Section
# III-A, equations F-interpolate and xjbar) on the same workload.
CURVES = [("p256", 1, 100, 10, 0.5, 0.5, 1.25)] + [
    ("p256", 1, 100, 10, a, 0.5, k) for a in (0.5, 2.0, 8.0) for k in (1.25, 2.0) if (a, k) != (0.5, 1.25)]


# (workload, seed, iterations, every, alpha, rho, kappa, perturbation): the
# bench's parameters under rounding-sized perturbations (see above).
SPREAD = [CURVES[0] + (p,) for p in ("in32", "in32_state32", "in32_fft32")]


def _fft2o_32(a):
    return np.fft.fft2(a.astype(np.complex64), norm="ortho").astype(np.complex128)


def _ifft2o_32(a):
    return np.fft.ifft2(a.astype(np.complex64), norm="ortho").astype(np.complex128)


def out_name(spec):
    name, _, _, _, alpha, _, kappa = spec[:7]
    if len(spec) == 8:
        return f"nrmse_{name}_spread_{spec[7]}.json"
    return f"nrmse_{name}.json" if spec == CURVES[0] else f"nrmse_{name}_a{alpha:g}_k{kappa:g}.json"


def curve(name, seed, iters, every, alpha, rho, kappa, perturbation=None):
    w = datagen.make_workload(name, seed=seed)
    mask = orc.weight_image(w.probe, w.offsets, w.x.shape, kappa) > 0
    probe, y = w.probe, w.y
    if perturbation in ("in32", "in32_state32", "in32_fft32"):
        probe = w.probe.astype(np.complex64).astype(np.complex128)
        y = w.y.astype(np.float32).astype(np.float64)
    elif perturbation is not None:
        raise ValueError(perturbation)
    if perturbation == "in32_fft32":   # this process only (one spawned process per curve)
        orc.fft2o, orc.ifft2o = _fft2o_32, _ifft2o_32
    state32 = perturbation == "in32_state32"
    step = 1 if state32 else every
    v = z = None
    points = []
    for k in range(step, iters + 1, step):
        o = orc.pmace(y, probe, w.offsets, w.x.shape, alpha=alpha, rho=rho, kappa=kappa,
                      n_iter=step, v0=v, z_prev=z)
        v, z = o["v"], o["z"]
        if state32:
            v = v.astype(np.complex64).astype(np.complex128)
            z = z.astype(np.complex64).astype(np.complex128)
        if k % every == 0:
            points.append(dict(iteration=k, nrmse=orc.nrmse(o["x_hat"], w.x, mask), r_fp=o["r_fp"],
                               r_data=o["r_data"]))
            print(name, perturbation or "", points[-1], flush=True)
    d = dict(workload=name, seed=seed, alpha=alpha, rho=rho, kappa=kappa,
             start="energy-matched constant", points=points)
    if perturbation is not None:
        d["perturbation"] = perturbation
    return d


def write(spec):
    d = curve(*spec)
    with open(os.path.join(HERE, out_name(spec)), "w") as f:
        json.dump(d, f, indent=1)


if __name__ == "__main__":
    # independent runs, one process each; `--only-missing` skips stored curves
    import multiprocessing as mp
    todo = [c for c in CURVES + SPREAD
            if "--only-missing" not in sys.argv or not os.path.exists(os.path.join(HERE, out_name(c)))]
    with mp.get_context("spawn").Pool(min(len(todo), os.cpu_count() or 1)) as pool:
        pool.map(write, todo)
