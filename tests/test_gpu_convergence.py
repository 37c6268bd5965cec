"""End-to-end reconstruction quality against the FP64 oracle's error curve.

The 600 x 600 / 256 x 256 / 324-window workload runs its full 100
iterations of Algorithm 1 from the energy-matched constant start; the NRMSE
of Section IV (global phase aligned, over the pixels some window covers) of
the GPU readout is compared with the oracle's at the same iteration counts,
stored in tests/golden/nrmse_p256.json by tests/golden/make_nrmse_curves.py
(which calls only the oracle).
"""
import json
import os

import numpy as np
import pytest

from oracle import pmace_oracle as orc
from paper_2111_14240_gb300 import datagen
from tests.gpu_helpers import TOL_NRMSE_REL, rounded_inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "nrmse_p256.json")


@pytest.mark.gpu
def test_p256_nrmse_curve_matches_oracle():
    from paper_2111_14240_gb300 import build
    from paper_2111_14240_gb300 import pmace as pm
    build.build()
    with open(GOLDEN) as f:
        g = json.load(f)
    w = datagen.make_workload(g["workload"], seed=g["seed"])
    _, _, probe32, y32 = rounded_inputs(w)
    mask = orc.weight_image(w.probe, w.offsets, w.x.shape, g["kappa"]) > 0
    rec = pm.Reconstruction(probe32, w.offsets, y32, w.x.shape, kappa=g["kappa"])
    try:
        done = 0
        for pt in g["points"]:
            rec.iterate(pt["iteration"] - done, g["alpha"], g["rho"])
            done = pt["iteration"]
            e = orc.nrmse(rec.image().cpu().numpy().astype(np.complex128), w.x, mask)
            print(f"p256 iteration {done}: NRMSE GPU {e:.5f} oracle {pt['nrmse']:.5f}")
            pt["gpu"] = e
    finally:
        rec.close()
    final = g["points"][-1]
    assert abs(final["gpu"] - final["nrmse"]) <= TOL_NRMSE_REL * final["nrmse"]
    # the GPU run also improves the reconstruction as the oracle's does
    assert final["gpu"] < g["points"][0]["gpu"]


def test_golden_curve_is_the_configured_run():
    """The stored curve is the generator's configuration (no GPU needed)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_nrmse_curves", os.path.join(os.path.dirname(GOLDEN), "make_nrmse_curves.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with open(GOLDEN) as f:
        g = json.load(f)
    name, seed, iters, every, alpha, rho, kappa = mod.CURVES[0]
    assert (g["workload"], g["seed"], g["alpha"], g["rho"], g["kappa"]) == (name, seed, alpha, rho, kappa)
    assert [p["iteration"] for p in g["points"]] == list(range(every, iters + 1, every))
    assert all(np.isfinite(p["nrmse"]) and p["nrmse"] > 0 for p in g["points"])
