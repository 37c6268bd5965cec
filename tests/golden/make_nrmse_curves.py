"""Write the FP64 oracle's reconstruction-error curves used by the GPU tests.

Runs Algorithm 1 of the oracle (and nothing else) on seeded synthetic
workloads from the energy-matched constant start and records the NRMSE of
Section IV (global phase aligned, over the pixels some window covers) of
the readout x_hat after every `every` iterations.  Usage:

    python tests/golden/make_nrmse_curves.py

writes tests/golden/nrmse_<name>[_a<alpha>_k<kappa>].json.  Deterministic:
the workloads come from seeded generators and the oracle is plain FP64 numpy.
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


def out_name(spec):
    name, _, _, _, alpha, _, kappa = spec
    return f"nrmse_{name}.json" if spec == CURVES[0] else f"nrmse_{name}_a{alpha:g}_k{kappa:g}.json"


def curve(name, seed, iters, every, alpha, rho, kappa):
    w = datagen.make_workload(name, seed=seed)
    mask = orc.weight_image(w.probe, w.offsets, w.x.shape, kappa) > 0
    v = z = None
    points = []
    for k in range(every, iters + 1, every):
        o = orc.pmace(w.y, w.probe, w.offsets, w.x.shape, alpha=alpha, rho=rho, kappa=kappa,
                      n_iter=every, v0=v, z_prev=z)
        v, z = o["v"], o["z"]
        points.append(dict(iteration=k, nrmse=orc.nrmse(o["x_hat"], w.x, mask), r_fp=o["r_fp"],
                           r_data=o["r_data"]))
        print(name, points[-1], flush=True)
    return dict(workload=name, seed=seed, alpha=alpha, rho=rho, kappa=kappa,
                start="energy-matched constant", points=points)


def write(spec):
    d = curve(*spec)
    with open(os.path.join(HERE, out_name(spec)), "w") as f:
        json.dump(d, f, indent=1)


if __name__ == "__main__":
    # independent runs, one process each; `--only-missing` skips stored curves
    import multiprocessing as mp
    todo = [c for c in CURVES if "--only-missing" not in sys.argv or not os.path.exists(os.path.join(HERE, out_name(c)))]
    with mp.get_context("spawn").Pool(min(len(todo), os.cpu_count() or 1)) as pool:
        pool.map(write, todo)
