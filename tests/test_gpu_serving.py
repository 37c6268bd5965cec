"""Serving loop: continuous batching of jobs of different sizes.

The same jobs are run (a) all submitted at once, so their windows share
launches, (b) one at a time through the server, and (c) through the plain
single-job API; every job's image must be identical bit for bit in all
three, and the budget-limited admission must still complete every job.
"""
import numpy as np
import pytest

from paper_2111_14240_gb300 import datagen
from tests.gpu_helpers import rounded_inputs

pytestmark = pytest.mark.gpu

# (object side, probe, sigma, raster n, step, jitter, iterations, fp16)
JOBS = [(96, 32, 8.0, 9, 8, 1, 7, False),
        (128, 32, 8.0, 13, 8, 1, 5, True),
        (160, 64, 16.0, 7, 16, 2, 9, False),
        (200, 64, 16.0, 9, 16, 2, 4, True),
        (300, 128, 32.0, 6, 32, 2, 6, False),
        (140, 32, 8.0, 10, 12, 1, 0, False)]


@pytest.fixture(scope="module")
def jobs():
    from paper_2111_14240_gb300 import build
    build.build()
    out = []
    for k, (side, n_p, sig, n_scan, step, jit, iters, f16) in enumerate(JOBS):
        cfg = dict(n_obj=side, n_p=n_p, probe_sigma=sig, n_scan=n_scan, step=step, jitter=jit,
                   peak=1e5, name=f"job{k}")
        w = datagen.make_workload(cfg, seed=100 + k)
        _, _, probe32, y32 = rounded_inputs(w)
        if f16:
            codes, scales = datagen.quantize_amplitudes_f16(y32.astype(np.float64))
            amps, sc = codes, scales
        else:
            amps, sc = y32, None
        out.append(dict(w=w, probe=probe32, amps=amps, scales=sc, iters=iters, f16=f16,
                        alpha=0.3 + 0.1 * k, rho=0.5 if k % 2 == 0 else 0.4))
    return out


def _submit(srv, pm, j):
    w = j["w"]
    return srv.submit(j["probe"], w.offsets, j["amps"], w.x.shape, j["iters"], j["alpha"], j["rho"],
                      amp_format=pm.PMACE_AMP_F16_SCALED if j["f16"] else pm.PMACE_AMP_F32,
                      scales=j["scales"])


def _plain(pm, j):
    import torch
    w = j["w"]
    if j["f16"]:
        rec = pm.Reconstruction(j["probe"], w.offsets, torch.from_numpy(j["amps"]).cuda(), w.x.shape,
                                amp_format=pm.PMACE_AMP_F16_SCALED,
                                scales=torch.from_numpy(j["scales"]).cuda())
    else:
        rec = pm.Reconstruction(j["probe"], w.offsets, j["amps"], w.x.shape)
    rec.iterate(j["iters"], j["alpha"], j["rho"])
    img = rec.image().cpu().numpy()
    rec.close()
    return img


def test_mixed_alone_and_plain_are_identical(jobs):
    from paper_2111_14240_gb300 import pmace as pm
    srv = pm.Server()
    ids = [_submit(srv, pm, j) for j in jobs]
    mixed = []
    for jid in ids:
        res, img = srv.wait(jid)
        assert res["done"] == 1 and res["status"] == 0, res
        mixed.append(img)
        srv.release(jid)
    st = srv.stats()
    assert st["completed"] == len(jobs) and st["queued"] == 0 and st["active"] == 0
    alone = []
    for j in jobs:
        jid = _submit(srv, pm, j)
        res, img = srv.wait(jid)
        assert res["status"] == 0
        alone.append(img)
    srv.close()
    for k, j in enumerate(jobs):
        plain = _plain(pm, j)
        assert np.array_equal(mixed[k], alone[k]), f"job {k}: mixed differs from alone"
        assert np.array_equal(mixed[k], plain), f"job {k}: server differs from the single-job API"


def test_budget_limited_admission_completes_everything(jobs):
    from paper_2111_14240_gb300 import pmace as pm
    # room for about one of the larger jobs at a time
    srv = pm.Server(hbm_budget_bytes=64 << 20, max_active_jobs=2)
    ids = [_submit(srv, pm, j) for j in jobs]
    imgs = []
    for jid in ids:
        res, img = srv.wait(jid)
        assert res["status"] == 0, res
        assert res["start_ms"] >= res["submit_ms"] and res["finish_ms"] >= res["start_ms"]
        imgs.append(img)
    srv.close()
    for k, j in enumerate(jobs):
        assert np.array_equal(imgs[k], _plain(pm, j))


def test_job_larger_than_budget_is_rejected(jobs):
    from paper_2111_14240_gb300 import pmace as pm
    srv = pm.Server(hbm_budget_bytes=1 << 20)
    jid = _submit(srv, pm, jobs[4])
    res, img = srv.wait(jid)
    assert res["done"] == 1 and res["status"] == pm.PMACE_ERR_OOM and img is None
    srv.close()


def test_wait_times_out_without_stopping_the_job(jobs):
    from paper_2111_14240_gb300 import pmace as pm
    srv = pm.Server()
    j = dict(jobs[2], iters=400)
    jid = _submit(srv, pm, j)
    with pytest.raises(pm.PmaceError) as e:
        srv.wait(jid, timeout_ms=1)
    assert e.value.status == pm.PMACE_ERR_TIMEOUT
    res, img = srv.wait(jid)
    assert res["status"] == 0 and img is not None
    srv.close()


def test_gave_up_wait_reaches_the_served_result_and_host_readout(jobs, monkeypatch):
    """A job whose error word records a device-side wait that gave up is
    retired with PMACE_ERR_TIMEOUT instead of an image, and a plain job's
    host readout and residual report it too.  The error word is set on the
    host at job creation (fault injection, PMACE_INJECT_WAIT_TIMEOUT); no
    device-side wait runs out."""
    import torch

    from paper_2111_14240_gb300 import pmace as pm
    monkeypatch.setenv("PMACE_INJECT_WAIT_TIMEOUT", "1")
    srv = pm.Server()
    jid = _submit(srv, pm, jobs[0])
    res, img = srv.wait(jid)
    srv.close()
    assert res["done"] == 1 and res["status"] == pm.PMACE_ERR_TIMEOUT and img is None
    j = jobs[2]
    rec = pm.Reconstruction(j["probe"], j["w"].offsets, j["amps"], j["w"].x.shape)
    try:
        rec.iterate(2, j["alpha"], j["rho"])
        rec.image()   # device readout: asynchronous, does not check
        host = np.empty(j["w"].x.shape, np.complex64)
        with pytest.raises(pm.PmaceError) as e:
            pm.pmace_get_image(rec.h, host)
        assert e.value.status == pm.PMACE_ERR_TIMEOUT
        with pytest.raises(pm.PmaceError) as e:
            rec.residual()
        assert e.value.status == pm.PMACE_ERR_TIMEOUT
        torch.cuda.synchronize()
    finally:
        rec.close()
    monkeypatch.delenv("PMACE_INJECT_WAIT_TIMEOUT")
    # a job created without the injection is unaffected
    assert np.isfinite(_plain(pm, jobs[0])).all()
