"""End-to-end reconstruction quality against the FP64 oracle's error curves.

The 600 x 600 / 256 x 256 / 324-window workload runs its full 100
iterations of Algorithm 1 from the energy-matched constant start, at the
bench's parameters and over a sweep of alpha and kappa.  The NRMSE of
Section IV (global phase aligned, over the pixels some window covers) of
the GPU readout is compared with the oracle's at the same iteration counts,
stored in tests/golden/nrmse_p256*.json by tests/golden/make_nrmse_curves.py
(which calls only the oracle).

The run at the bench's parameters does not settle within 100 iterations
(the oracle's fixed-point residual is still near 1 there), and its error
curve moves by a few percent under rounding alone: the FP64 oracle fed the
inputs rounded to single precision, exactly as the GPU receives them, ends
3 % away from the FP64-input run.  Those perturbed oracle runs are stored
beside the curves (nrmse_p256_spread_*.json: single-precision inputs, plus
single-precision state or single-precision FFTs), and the bar is taken
against them, at the first stored count and at the final one: the larger
of 1 % and twice the largest move of a perturbed run there.  The counts in
between are not held point by point: how far two runs that differ only in
rounding sit apart there swings from one count to the next.
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
CURVE_FILES = [p for p in sorted(glob.glob(os.path.join(GOLDEN_DIR, "nrmse_p256*.json"))) if "_spread_" not in p]
SPREAD_FILES = sorted(glob.glob(os.path.join(GOLDEN_DIR, "nrmse_p256_spread_*.json")))
# At the first stored count the perturbed oracle runs must still agree with
# the oracle to well within the 1 % bar, so that the bar holds there.
TIGHT_SPREAD = TOL_NRMSE_REL / 4


def _generator():
    spec = importlib.util.spec_from_file_location("make_nrmse_curves",
                                                  os.path.join(GOLDEN_DIR, "make_nrmse_curves.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _load(path):
    with open(path) as f:
        return json.load(f)


def oracle_spread():
    """Per stored iteration count of the bench-parameter curve, the largest
    relative distance of a rounding-perturbed oracle run from the oracle."""
    ref = [pt["nrmse"] for pt in _load(os.path.join(GOLDEN_DIR, "nrmse_p256.json"))["points"]]
    spread = [0.0] * len(ref)
    for path in SPREAD_FILES:
        pts = [pt["nrmse"] for pt in _load(path)["points"]]
        assert len(pts) == len(ref), path
        spread = [max(s, abs(p - r) / r) for s, p, r in zip(spread, pts, ref)]
    return spread


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
    spread = oracle_spread()
    # the first and the final stored counts: 1 % or twice the oracle's own
    # rounding spread there, whichever is larger
    for i in (0, len(ref) - 1):
        bar = max(TOL_NRMSE_REL, 2.0 * spread[i])
        assert abs(got[i] - ref[i]) <= bar * ref[i], (g["points"][i]["iteration"], got[i], ref[i], bar)
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
    for spec in mod.CURVES + mod.SPREAD:
        path = os.path.join(GOLDEN_DIR, mod.out_name(spec))
        assert os.path.exists(path), path
        g = _load(path)
        name, seed, iters, every, alpha, rho, kappa = spec[:7]
        assert (g["workload"], g["seed"], g["alpha"], g["rho"], g["kappa"]) == (name, seed, alpha, rho, kappa)
        assert g.get("perturbation") == (spec[7] if len(spec) == 8 else None)
        assert [p["iteration"] for p in g["points"]] == list(range(every, iters + 1, every))
        assert all(np.isfinite(p["nrmse"]) and p["nrmse"] > 0 for p in g["points"])
    assert sorted(SPREAD_FILES) == sorted(os.path.join(GOLDEN_DIR, mod.out_name(s)) for s in mod.SPREAD)


def test_oracle_spread_is_rounding_sized():
    """The perturbed runs start close to the oracle (they differ by rounding
    only), so the bar at the first stored count is the plain 1 % (no GPU)."""
    spread = oracle_spread()
    assert spread[0] <= TIGHT_SPREAD
    assert max(TOL_NRMSE_REL, 2.0 * spread[0]) == TOL_NRMSE_REL
