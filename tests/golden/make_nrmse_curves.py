"""Write the FP64 oracle's reconstruction-error curves used by the GPU tests.

Runs Algorithm 1 of the oracle (and nothing else) on seeded synthetic
workloads from the energy-matched constant start and records, after every
`every` iterations, the NRMSE of Section IV (global phase aligned) of the
readout x_hat over two pixel masks:

  nrmse      the pixels some window covers (Lambda > 0);
  nrmse_lit  the well-illuminated pixels, Lambda >= LIT_FRACTION max Lambda
             (Lambda = sum_j P_j^t |D|^kappa, Section III-A, equation
             xjbar): where the summed probe weight is a tenth of its peak or
             more.  Pixels at the edge of a scan are seen only through the
             tails of the probe; there D^-1 amplifies the data term by up to
             1/|d| and the reconstruction is not determined by the data.

Usage:

    python tests/golden/make_nrmse_curves.py [--only-missing]

Deterministic: the workloads come from seeded generators and the oracle is
plain FP64 numpy.  Two groups of curves:

* the 600 x 600 / 256 x 256 / 324-window workload at the bench's parameters
  and over an alpha / kappa sweep (nrmse_p256*.json);
* a geometry that converges, the 128 x 128 probe (sigma 32 px) raster of the
  2048 x 2048 workload (step 16 px, +-2 px jitter) on a 30 x 30 scan of a
  600 x 600 object, at Poisson peaks 1e4 and 1e6 and alpha 0.5 and 2
  (nrmse_c30_*.json), and the 128 x 128 / 32 x 32 / 169-window workload at
  peak 1e5 for its 50 iterations (nrmse_small_*.json).

Beside the bench-parameter curve and the alpha = 0.5 curves of the
converging geometry it writes the same oracle run under perturbations of
the size of single-precision rounding (<curve>_spread_<perturbation>.json),
which measure how far the oracle's own error curve moves when nothing but
rounding changes:

  in32          the probe rounded to complex64 and the amplitudes to float32
                (the inputs exactly as the GPU receives them);
  in32_state32  the same inputs, and the carried state (the stack v and the
                consensus stack z) rounded to complex64 after every
                iteration, as single-precision storage would;
  in32_fft32    the same inputs, and the oracle's two transforms (fft2o,
                ifft2o) evaluated in single precision (numpy's complex64
                FFT), everything else in FP64;
  in32_all32    the same inputs, and every step of Algorithm 1 in single
                precision (complex64 transforms, agent arithmetic, consensus
                sums and state, float32 weights), in the oracle's order: the
                arithmetic precision the hot path is specified to use;
  in32_ulpS     (bench-parameter curve only, S = 1 .. 6) the in32 inputs with
                every amplitude and every real and imaginary part of the
                probe moved by one single-precision unit of relative size
                2^-24, up or down at random (seed S), then the plain FP64
                oracle: an ensemble of equally sized rounding changes, which
                samples how far rounding alone moves a curve that does not
                converge.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "..", ".."))

from oracle import pmace_oracle as orc  # noqa: E402
from paper_2111_14240_gb300 import datagen  # noqa: E402

LIT_FRACTION = 0.1

# the converging geometry: 128 x 128 probe raster of the 2048 x 2048 workload
C30 = dict(n_obj=600, n_p=128, probe_sigma=32.0, n_scan=30, step=16, jitter=2, name="c30")

PERTURBATIONS = ("in32", "in32_state32", "in32_fft32", "in32_all32")
ULP_SEEDS = (1, 2, 3, 4, 5, 6)


def _spec(group, workload, seed, iters, every, alpha, kappa, peak=None, perturbation=None, rho=0.5):
    return dict(group=group, workload=workload, seed=seed, iters=iters, every=every, alpha=alpha,
                rho=rho, kappa=kappa, peak=peak, perturbation=perturbation)


# (a) 600 x 600 / 256 x 256 / 324 windows: the bench's parameters, then the
# sweep of the noise-to-signal ratio alpha and the probe exponent kappa
# (Section III-A, equations F-interpolate and xjbar)
CURVES = [_spec("p256", "p256", 1, 100, 10, 0.5, 1.25)] + [
    _spec("p256", "p256", 1, 100, 10, a, k) for a in (0.5, 2.0, 8.0) for k in (1.25, 2.0)
    if (a, k) != (0.5, 1.25)]
# (b) the converging geometry at two photon peaks and two alphas, and the
# 169-window workload
CURVES += [_spec("c30", "c30", 1, 100, 10, a, 1.25, peak=pk) for pk in (1e4, 1e6) for a in (0.5, 2.0)]
CURVES += [_spec("small", "small", 1, 50, 5, a, 1.25) for a in (0.5, 2.0)]

# the rounding-sized perturbations of the bench-parameter curve and of the
# alpha = 0.5 curves of the converging geometry
SPREAD = [dict(CURVES[0], perturbation=p) for p in PERTURBATIONS]
SPREAD += [dict(CURVES[0], perturbation=f"in32_ulp{k}") for k in ULP_SEEDS]
SPREAD += [dict(c, perturbation=p) for c in CURVES if c["group"] == "c30" and c["alpha"] == 0.5
           for p in ("in32", "in32_all32")]


def out_name(spec):
    """File name of a curve: nrmse_p256.json for the bench-parameter run,
    nrmse_p256_a<alpha>_k<kappa>.json for the sweep,
    nrmse_c30_pk<peak>_a<alpha>.json, nrmse_small_a<alpha>.json, and
    <base>_spread_<perturbation>.json for the perturbed runs."""
    g = spec["group"]
    if g == "p256":
        base = ("nrmse_p256" if (spec["alpha"], spec["kappa"]) == (0.5, 1.25)
                else f"nrmse_p256_a{spec['alpha']:g}_k{spec['kappa']:g}")
    elif g == "c30":
        base = f"nrmse_c30_pk{spec['peak']:.0e}_a{spec['alpha']:g}".replace("+0", "")
    else:
        base = f"nrmse_{g}_a{spec['alpha']:g}"
    if spec["perturbation"]:
        base += f"_spread_{spec['perturbation']}"
    return base + ".json"


def workload(spec):
    """The seeded workload of a curve (datagen only)."""
    cfg = C30 if spec["workload"] == "c30" else spec["workload"]
    if spec["peak"] is None:
        return datagen.make_workload(cfg, seed=spec["seed"])
    return datagen.make_workload(cfg, seed=spec["seed"], peak=spec["peak"])


def masks(w, kappa):
    """The covered pixels (Lambda > 0) and the well-illuminated ones
    (Lambda >= LIT_FRACTION max Lambda)."""
    lam = orc.weight_image(w.probe, w.offsets, w.x.shape, kappa)
    return lam > 0, lam >= LIT_FRACTION * lam.max()


def _fft2o_32(a):
    return np.fft.fft2(a.astype(np.complex64), norm="ortho").astype(np.complex128)


def _ifft2o_32(a):
    return np.fft.ifft2(a.astype(np.complex64), norm="ortho").astype(np.complex128)


def _pmace_all32(y, probe, offsets, shape, alpha, rho, kappa, n_iter, v0=None, z_prev=None):
    """Algorithm 1 in the oracle's order with every array in single
    precision: w <- F(v) (complex64 transforms and agent arithmetic), z <-
    G(2w - v) (float32 weights, complex64 sums), v <- v + 2 rho (z - w).
    Returns (v, z, x_hat) in complex128."""
    c64 = np.complex64
    n_p = probe.shape[0]
    d = probe.astype(c64)
    y32 = y.astype(np.float32)
    lam_inv = orc.inverse_weights(orc.weight_image(probe, offsets, shape, kappa)).astype(np.float32)
    wk = (np.abs(probe) ** kappa).astype(np.float32)
    ok = np.abs(probe) > orc.TINY_PROBE * np.abs(probe).max()
    if v0 is None:
        v = orc.init_stack(orc.default_init(y, probe, shape), offsets, n_p).astype(c64)
    else:
        v = v0.astype(c64)
    z = v.copy() if z_prev is None else z_prev.astype(c64)

    def consensus_image(stack):
        img = np.zeros(shape, dtype=c64)
        for i, (r, c) in enumerate(offsets):
            img[r:r + n_p, c:c + n_p] += wk * stack[i]
        return img * lam_inv

    for _ in range(n_iter):
        a = np.fft.fft2(d[None] * v, norm="ortho")
        mag = np.abs(a)
        ph = np.zeros_like(a)
        np.divide(a, mag, out=ph, where=mag > 0)
        back = np.fft.ifft2(y32 * ph, norm="ortho")
        data = np.zeros_like(back)
        np.divide(back, d[None], out=data, where=ok[None])
        w = np.where(ok[None], (alpha * v + data) / np.float32(1.0 + alpha), v).astype(c64)
        xbar = consensus_image(2 * w - v)
        z = np.stack([xbar[r:r + n_p, c:c + n_p] for r, c in offsets])
        v = (v + np.float32(2.0 * rho) * (z - w)).astype(c64)
    x_hat = consensus_image(v)
    return v.astype(np.complex128), z.astype(np.complex128), x_hat.astype(np.complex128)


def curve(spec):
    w = workload(spec)
    alpha, rho, kappa = spec["alpha"], spec["rho"], spec["kappa"]
    iters, every, pert = spec["iters"], spec["every"], spec["perturbation"]
    cover, lit = masks(w, kappa)
    probe, y = w.probe, w.y
    if pert is not None:
        ulp_seed = int(pert[len("in32_ulp"):]) if pert.startswith("in32_ulp") else None
        if pert not in PERTURBATIONS and ulp_seed not in ULP_SEEDS:
            raise ValueError(pert)
        probe = w.probe.astype(np.complex64).astype(np.complex128)
        y = w.y.astype(np.float32).astype(np.float64)
        if ulp_seed is not None:
            rng = np.random.Generator(np.random.PCG64(1000 + ulp_seed))
            eps = 2.0 ** -24
            y = y * (1.0 + eps * rng.choice((-1.0, 1.0), size=y.shape))
            probe = (probe.real * (1.0 + eps * rng.choice((-1.0, 1.0), size=probe.shape))
                     + 1j * probe.imag * (1.0 + eps * rng.choice((-1.0, 1.0), size=probe.shape)))
    if pert == "in32_fft32":   # this process only (one spawned process per curve)
        orc.fft2o, orc.ifft2o = _fft2o_32, _ifft2o_32
    state32 = pert == "in32_state32"
    step = 1 if state32 else every
    v = z = None
    points = []
    for k in range(step, iters + 1, step):
        if pert == "in32_all32":
            v, z, x_hat = _pmace_all32(y, probe, w.offsets, w.x.shape, alpha, rho, kappa, step, v, z)
            r_fp = r_data = None
        else:
            o = orc.pmace(y, probe, w.offsets, w.x.shape, alpha=alpha, rho=rho, kappa=kappa,
                          n_iter=step, v0=v, z_prev=z)
            v, z, x_hat, r_fp, r_data = o["v"], o["z"], o["x_hat"], o["r_fp"], o["r_data"]
        if state32:
            v = v.astype(np.complex64).astype(np.complex128)
            z = z.astype(np.complex64).astype(np.complex128)
        if k % every == 0:
            points.append(dict(iteration=k, nrmse=orc.nrmse(x_hat, w.x, cover),
                               nrmse_lit=orc.nrmse(x_hat, w.x, lit), r_fp=r_fp, r_data=r_data))
            print(out_name(spec), points[-1], flush=True)
    d = dict(workload=spec["workload"], seed=spec["seed"], alpha=alpha, rho=rho, kappa=kappa,
             peak=w.peak, start="energy-matched constant", lit_fraction=LIT_FRACTION,
             lit_pixels=int(lit.sum()), cover_pixels=int(cover.sum()), points=points)
    if pert is not None:
        d["perturbation"] = pert
    return d


def write(spec):
    d = curve(spec)
    with open(os.path.join(HERE, out_name(spec)), "w") as f:
        json.dump(d, f, indent=1)


if __name__ == "__main__":
    # independent runs, one process each (spawned); `--only-missing` skips
    # stored curves; `--group <g>` restricts to one group
    import multiprocessing as mp
    todo = CURVES + SPREAD
    if "--group" in sys.argv:
        g = sys.argv[sys.argv.index("--group") + 1]
        todo = [c for c in todo if c["group"] == g]
    if "--only-missing" in sys.argv:
        todo = [c for c in todo if not os.path.exists(os.path.join(HERE, out_name(c)))]
    # longest runs first
    todo.sort(key=lambda c: -(c["iters"] * (4 if c["group"] == "p256" else 1)))
    with mp.get_context("spawn").Pool(min(len(todo), os.cpu_count() or 1)) as pool:
        pool.map(write, todo, chunksize=1)
