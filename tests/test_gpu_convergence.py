"""End-to-end reconstruction quality against the FP64 oracle's error curves.

The 600 x 600 / 256 x 256 / 324-window workload runs its full 100
iterations of Algorithm 1 from the energy-matched constant start, at the
bench's parameters and over a sweep of alpha and kappa.  The NRMSE of
Section IV (global phase aligned, over the pixels some window covers) of
the GPU readout is compared with the oracle's at the same iteration counts,
stored in tests/golden/nrmse_p256*.json by tests/golden/make_nrmse_curves.py
(which calls only the oracle).
"""
import glob
import importlib.util
import json
import os

import numpy as np
import pytest

from oracle import pmace_oracle as orc
from paper_2111_14240_gb300 import datagen
from tests.gpu_helpers import TOL_NRMSE_REL, rounded_inputs

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
CURVE_FILES = sorted(glob.glob(os.path.join(GOLDEN_DIR, "nrmse_p256*.json")))


def _generator():
    spec = importlib.util.spec_from_file_location("make_nrmse_curves",
                                                  os.path.join(GOLDEN_DIR, "make_nrmse_curves.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def gpu_curve(g):
    """NRMSE of the GPU readout at the stored curve's iteration counts."""
    from paper_2111_14240_gb300 import pmace as pm
    w = datagen.make_workload(g["workload"], seed=g["seed"])
    _, _, probe32, y32 = rounded_inputs(w)
    mask = orc.weight_image(w.probe, w.offsets, w.x.shape, g["kappa"]) > 0
    rec = pm.Reconstruction(probe32, w.offsets, y32, w.x.shape, kappa=g["kappa"])
    out = []
    try:
        done = 0
        for pt in g["points"]:
            rec.iterate(pt["iteration"] - done, g["alpha"], g["rho"])
            done = pt["iteration"]
            out.append(orc.nrmse(rec.image().cpu().numpy().astype(np.complex128), w.x, mask))
    finally:
        rec.close()
    return out


# The alpha / kappa sweep on this poorly illuminated geometry: FP32 and FP64
# trajectories separate by a few percent (pixels at the scan edge see 1e-2 to
# 1e-3 of the probe peak, and 1/d amplifies their data term), so the sweep is
# held to the ranking of the grid and 5 % on the final error; the bench's own
# parameters keep the 1 % bar.
TOL_SWEEP_REL = 0.05


@pytest.fixture(scope="module")
def curves():
    from paper_2111_14240_gb300 import build
    build.build()
    out = []
    for path in CURVE_FILES:
        with open(path) as f:
            g = json.load(f)
        got = gpu_curve(g)
        for pt, e in zip(g["points"], got):
            print(f"p256 alpha={g['alpha']} kappa={g['kappa']} iteration {pt['iteration']}: "
                  f"NRMSE GPU {e:.5f} oracle {pt['nrmse']:.5f}")
        out.append((g, got))
    return out


@pytest.mark.gpu
def test_p256_nrmse_at_bench_parameters(curves):
    g, got = next(c for c in curves if (c[0]["alpha"], c[0]["kappa"]) == (0.5, 1.25))
    ref = [pt["nrmse"] for pt in g["points"]]
    assert abs(got[-1] - ref[-1]) <= TOL_NRMSE_REL * ref[-1]
    # the GPU run moves the error the same way over the run as the oracle's
    assert (got[-1] < got[0]) == (ref[-1] < ref[0])


@pytest.mark.gpu
def test_p256_alpha_kappa_sweep(curves):
    for g, got in curves:
        ref = [pt["nrmse"] for pt in g["points"]]
        assert abs(got[-1] - ref[-1]) <= TOL_SWEEP_REL * ref[-1], (g["alpha"], g["kappa"], got[-1], ref[-1])
        assert (got[-1] < got[0]) == (ref[-1] < ref[0])
    # the grid's ranking: every pair the oracle separates by more than 10 %
    # comes out in the same order on the GPU
    fin_o = [c[0]["points"][-1]["nrmse"] for c in curves]
    fin_g = [c[1][-1] for c in curves]
    for i in range(len(curves)):
        for k in range(len(curves)):
            if fin_o[i] * 1.1 < fin_o[k]:
                assert fin_g[i] < fin_g[k]


def test_golden_curves_are_the_configured_runs():
    """Every configured curve is stored and is the generator's configuration (no GPU needed)."""
    mod = _generator()
    for spec in mod.CURVES:
        path = os.path.join(GOLDEN_DIR, mod.out_name(spec))
        assert os.path.exists(path), path
        with open(path) as f:
            g = json.load(f)
        name, seed, iters, every, alpha, rho, kappa = spec
        assert (g["workload"], g["seed"], g["alpha"], g["rho"], g["kappa"]) == (name, seed, alpha, rho, kappa)
        assert [p["iteration"] for p in g["points"]] == list(range(every, iters + 1, every))
        assert all(np.isfinite(p["nrmse"]) and p["nrmse"] > 0 for p in g["points"])
