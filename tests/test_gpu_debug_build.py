"""The bounds-checking build of the library (compiled with -DPMACE_DEBUG
into libpmace_debug.so).  Its device-side checks (window corners inside the
image, window indices inside [0, J), gather units inside their tables)
clamp or skip an access that would leave a job's arrays and report it
through the job's error word as PMACE_ERR_STATE.  Checked here:

* on valid inputs it computes exactly what the release build computes (the
  checks never fire and do not change the arithmetic), for a 64 x 64 probe
  (the in-place cross-CTA plan) and a 128 x 128 probe (the exchange plan);
* a window corner corrupted on the device after the job was created (a
  host-side fault injection that only this build honours) is caught: the
  iteration completes, reads nothing outside the job's arrays, and the
  residual and the host readout report PMACE_ERR_STATE.

Each build runs in its own process (the binding loads one library).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
import numpy as np
from paper_2111_14240_gb300 import datagen
from paper_2111_14240_gb300 import pmace as pm
out = {"library": pm._LIB_PATH, "status": []}
imgs = []
for cfg in (dict(n_obj=200, n_p=64, probe_sigma=16.0, n_scan=9, step=16, jitter=2, peak=1e5, name="mid64"),
            dict(n_obj=400, n_p=128, probe_sigma=32.0, n_scan=9, step=32, jitter=2, peak=1e5, name="mid128")):
    w = datagen.make_workload(cfg, seed=3)
    rec = pm.Reconstruction(w.probe.astype(np.complex64), w.offsets, w.y.astype(np.float32), w.x.shape)
    rec.iterate(3, 0.5, 0.5)
    st = 0
    try:
        rec.residual()
        img = np.empty(w.x.shape, np.complex64)
        pm.pmace_get_image(rec.h, img)
        imgs.append(img)
    except pm.PmaceError as e:
        st = e.status
    out["status"].append(st)
    rec.close()
if imgs:
    np.save(sys.argv[1], np.concatenate([i.ravel() for i in imgs]))
print(json.dumps(out))
"""


def _run(tmp_path, name, library=None, inject=False):
    env = dict(os.environ)
    env.pop("PMACE_LIBRARY", None)
    env.pop("PMACE_INJECT_BAD_OFFSET", None)
    if library:
        env["PMACE_LIBRARY"] = library
    if inject:
        env["PMACE_INJECT_BAD_OFFSET"] = "1"
    path = str(tmp_path / f"{name}.npy")
    r = subprocess.run([sys.executable, "-c", SCRIPT, path], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    return res, (np.load(path) if os.path.exists(path) else None)


@pytest.fixture(scope="module")
def debug_library():
    from paper_2111_14240_gb300 import build
    build.build()
    return build.build_debug()


def test_debug_build_matches_release(debug_library, tmp_path):
    rel, img_rel = _run(tmp_path, "release")
    dbg, img_dbg = _run(tmp_path, "debug", library=debug_library)
    assert dbg["library"].endswith("libpmace_debug.so") and not rel["library"].endswith("libpmace_debug.so")
    assert rel["status"] == [0, 0] and dbg["status"] == [0, 0]
    assert np.array_equal(img_rel, img_dbg)


def test_debug_build_catches_corrupt_window_corner(debug_library, tmp_path):
    from paper_2111_14240_gb300 import pmace as pm
    res, _ = _run(tmp_path, "inject", library=debug_library, inject=True)
    assert res["status"] == [pm.PMACE_ERR_STATE, pm.PMACE_ERR_STATE]
