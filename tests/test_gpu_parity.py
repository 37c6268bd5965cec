"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Workloads follow the synthetic recipe of the generator (smoothed random
object, Gaussian probe with quadratic phase, jittered raster, Poisson
amplitudes); sizes are chosen so the oracle finishes in seconds while the
kernels still span several tiles, clusters and a ragged image tail.
"""
import numpy as np
import pytest

from paper_2111_14240_gb300 import datagen
from tests.gpu_helpers import (TOL_ITER, TOL_NRMSE_REL, fused_state, random_start, rel_l2,
                               rounded_inputs, run_gpu, run_oracle)

pytestmark = pytest.mark.gpu

# probe sizes 64 and 128 on smaller objects than the full configurations
MID64 = dict(n_obj=200, n_p=64, probe_sigma=16.0, n_scan=9, step=16, jitter=2, peak=1e5)
MID128 = dict(n_obj=400, n_p=128, probe_sigma=32.0, n_scan=9, step=32, jitter=2, peak=1e5)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    from paper_2111_14240_gb300 import build
    build.build()


def _weighted(v, probe):
    return v * np.abs(probe)[None]


def _check_iteration(w, iters=1, alpha=0.5, rho=0.5, variant=None, f16=False, tol=TOL_ITER):
    """Iterations from a well-conditioned random start (see random_start)."""
    x0 = random_start(w)
    g = run_gpu(w, iters, alpha, rho, variant=variant, f16=f16, init=x0)
    o = run_oracle(w, iters, alpha, rho, f16=f16, x0=x0)
    e_img = rel_l2(g["x_hat"], o["x_hat"])
    e_vw = rel_l2(_weighted(g["v"], w.probe), _weighted(o["v"], w.probe))
    e_v = rel_l2(g["v"], o["v"])
    print(f"{w.name} np={w.np_} J={w.J} plan={g['plan']} iters={iters}: "
          f"x_hat {e_img:.2e}  |d|v {e_vw:.2e}  v {e_v:.2e}")
    # the unweighted stack too: D^-1 multiplies the rounding of the
    # single-precision transforms by 1/|d| (rms 8 for the sigma = Np / 4
    # probes, 94 for the 256 x 256 probe with sigma 48 px), and the bar holds
    # for it on every workload here
    assert e_img < tol and e_vw < tol and e_v < tol
    return g, o


def test_one_iteration_small():
    w = datagen.make_workload("small", seed=1)
    _check_iteration(w, 1)


def test_five_iterations_small():
    w = datagen.make_workload("small", seed=2)
    g, o = _check_iteration(w, 5, alpha=0.3, rho=0.4)
    assert abs(g["r_fp"] - o["r_fp"]) < 1e-4 * o["r_fp"]
    assert abs(g["r_data"] - o["r_data"]) < 1e-4 * o["r_data"]


VARIANTS = [0, 1, 2, 3, 4]   # every compiled agent kernel variant of a probe size


@pytest.mark.parametrize("variant", VARIANTS)
def test_one_iteration_np32(variant):
    w = datagen.make_workload("small", seed=17)
    g, _ = _check_iteration(w, 1, variant=variant)
    assert g["plan"]["variant"] == variant


@pytest.mark.parametrize("variant", VARIANTS)
def test_one_iteration_np64(variant):
    w = datagen.make_workload(dict(MID64, name="mid64"), seed=3)
    g, _ = _check_iteration(w, 1, variant=variant)
    assert g["plan"]["variant"] == variant


@pytest.mark.parametrize("variant", VARIANTS + [5])
def test_one_iteration_np128(variant):
    w = datagen.make_workload(dict(MID128, name="mid128"), seed=4)
    g, _ = _check_iteration(w, 1, variant=variant)
    assert g["plan"]["variant"] == variant


@pytest.mark.parametrize("variant", VARIANTS)
def test_one_iteration_np256_full_config(variant):
    """The 600 x 600 / 256 x 256 / 324-window workload at full size."""
    w = datagen.make_workload("p256", seed=1)
    g, _ = _check_iteration(w, 1, variant=variant)
    assert g["plan"]["variant"] == variant


@pytest.mark.parametrize("cfg,wpc,variant", [("small", 4, 4), ("mid64", 5, 4), ("mid128", 7, 4), ("mid128", 6, 5),
                                              ("mid128", 2, 5)])
def test_exchange_variant_runs_of_windows(cfg, wpc, variant, monkeypatch):
    """The transposing-exchange variants with a fixed run of windows per
    cluster (the last run shorter; for the two-window variant the last run
    ends in a single window), three iterations: the per-slab barriers are
    re-armed window after window and iteration after iteration."""
    spec = {"small": "small", "mid64": dict(MID64, name="mid64"), "mid128": dict(MID128, name="mid128")}[cfg]
    w = datagen.make_workload(spec, seed=31)
    assert w.J % wpc != 0
    monkeypatch.setenv("PMACE_AGENT_WPC", str(wpc))
    g, _ = _check_iteration(w, 3, variant=variant)
    assert g["plan"]["exchange"] == (1 if variant == 4 else 2) and g["plan"]["windows_per_cluster"] == wpc


def _midrun_step(w, k, alpha=0.5, rho=0.5, variant=None):
    """One iteration from the FP64 oracle's state after k iterations from the
    energy-matched constant start (loaded through the checkpoint call)."""
    from oracle import pmace_oracle as orc
    o_k = run_oracle(w, k, alpha, rho)
    q, xb = fused_state(o_k, rho)
    q = q.astype(np.complex64).astype(np.complex128)
    xb = xb.astype(np.complex64).astype(np.complex128)
    z = orc.redistribute(xb, w.offsets, w.np_)
    o = run_oracle(w, 1, alpha, rho, v0=q + 2 * rho * z, z_prev=z)
    g = run_gpu(w, 1, alpha, rho, variant=variant, state=(q, xb, k, rho))
    e_img = rel_l2(g["x_hat"], o["x_hat"])
    e_vw = rel_l2(_weighted(g["v"], w.probe), _weighted(o["v"], w.probe))
    e_v = rel_l2(g["v"], o["v"])
    print(f"{w.name} np={w.np_} mid-run k={k} plan={g['plan']}: x_hat {e_img:.2e}  |d|v {e_vw:.2e}"
          f"  v {e_v:.2e}")
    assert e_img < TOL_ITER and e_vw < TOL_ITER and e_v < TOL_ITER
    assert abs(g["r_fp"] - o["r_fp"]) < 1e-4 * o["r_fp"]
    assert abs(g["r_data"] - o["r_data"]) < 1e-4 * o["r_data"]


def test_midrun_iteration_small():
    _midrun_step(datagen.make_workload("small", seed=14), 10)


def test_midrun_iteration_np128():
    _midrun_step(datagen.make_workload(dict(MID128, name="mid128"), seed=15), 5)


@pytest.mark.parametrize("variant", [0, 2, 4])
def test_midrun_iteration_np256_full_config(variant):
    _midrun_step(datagen.make_workload("p256", seed=3), 3, variant=variant)


def test_nrmse_from_constant_start_np128():
    """From the constant start (mostly sub-FP32 spectra at first) the run
    still reaches the oracle's reconstruction quality."""
    from oracle import pmace_oracle as orc
    w = datagen.make_workload(dict(MID128, name="mid128"), seed=16)
    g = run_gpu(w, 30, 0.5, 0.5, want_patches=False)
    o = run_oracle(w, 30, 0.5, 0.5)
    mask = orc.weight_image(w.probe, w.offsets, w.x.shape, 1.25) > 0
    eg, eo = orc.nrmse(g["x_hat"], w.x, mask), orc.nrmse(o["x_hat"], w.x, mask)
    print(f"mid128 NRMSE after 30 iterations: GPU {eg:.5f} oracle {eo:.5f}")
    assert abs(eg - eo) <= TOL_NRMSE_REL * eo


def test_nrmse_50_iterations_small():
    w = datagen.make_workload("small", seed=1)
    from oracle import pmace_oracle as orc
    g = run_gpu(w, 50, 0.5, 0.5, want_patches=False)
    o = run_oracle(w, 50, 0.5, 0.5)
    mask = orc.weight_image(w.probe, w.offsets, w.x.shape, 1.25) > 0
    eg = orc.nrmse(g["x_hat"], w.x, mask)
    eo = orc.nrmse(o["x_hat"], w.x, mask)
    print(f"NRMSE after 50 iterations: GPU {eg:.5f} oracle {eo:.5f}")
    assert abs(eg - eo) <= TOL_NRMSE_REL * eo


@pytest.mark.parametrize("cfg,iters", [("small", 2), (dict(MID64, name="mid64"), 1),
                                       (dict(MID128, name="mid128"), 1), ("p256", 1)],
                         ids=["np32", "np64", "np128", "np256"])
def test_f16_amplitudes(cfg, iters):
    """FP16 amplitudes with a per-pattern scale, on each probe size's default plan."""
    w = datagen.make_workload(cfg, seed=6)
    _check_iteration(w, iters, f16=True)


def test_deterministic_np256():
    w = datagen.make_workload("p256", seed=2)
    a = run_gpu(w, 3, 0.5, 0.5)
    b = run_gpu(w, 3, 0.5, 0.5)
    assert np.array_equal(a["x_hat"], b["x_hat"]) and np.array_equal(a["v"], b["v"])
    assert a["r_fp"] == b["r_fp"] and a["r_data"] == b["r_data"]


def test_checkpoint_resume_bit_exact():
    import torch

    from paper_2111_14240_gb300 import pmace as pm
    w = datagen.make_workload("small", seed=7)
    _, _, probe32, y32 = rounded_inputs(w)
    a = pm.Reconstruction(probe32, w.offsets, y32, w.x.shape)
    a.iterate(3, 0.5, 0.4)
    q = torch.empty((w.J, 32, 32, 2), device="cuda")
    xb = torch.empty((128, 128, 2), device="cuda")
    info = pm.pmace_get_state(a.h, q, xb)
    assert info.iterations == 3 and abs(info.rho_pending - 0.4) < 1e-7
    a.iterate(2, 0.5, 0.6)
    ref = a.image().cpu().numpy()
    b = pm.Reconstruction(probe32, w.offsets, y32, w.x.shape)
    pm.pmace_set_state(b.h, q, xb, info)
    b.iterate(2, 0.5, 0.6)
    got = b.image().cpu().numpy()
    assert np.array_equal(ref, got)
    assert a.residual() == b.residual()
    a.close()
    b.close()


def test_changing_rho_between_calls_matches_oracle():
    """The pending rho closes the previous Mann step with the rho it was opened with."""
    from oracle import pmace_oracle as orc
    w = datagen.make_workload("small", seed=8)
    probe64, y64, probe32, y32 = rounded_inputs(w)
    from paper_2111_14240_gb300 import pmace as pm
    rec = pm.Reconstruction(probe32, w.offsets, y32, w.x.shape)
    rec.iterate(2, 0.5, 0.3)
    rec.iterate(2, 0.7, 0.6)
    got = rec.image().cpu().numpy().astype(np.complex128)
    rec.close()
    r1 = orc.pmace(y64, probe64, w.offsets, w.x.shape, alpha=0.5, rho=0.3, n_iter=2)
    r2 = orc.pmace(y64, probe64, w.offsets, w.x.shape, alpha=0.7, rho=0.6, n_iter=2, v0=r1["v"],
                   z_prev=r1["z"])
    assert rel_l2(got, r2["x_hat"]) < TOL_ITER


def test_single_window_covers_image():
    """J = 1 with the window equal to the image: G is the identity."""
    rng = np.random.Generator(np.random.PCG64(9))
    x = datagen.make_object(rng, 64, 64)
    d = datagen.make_probe(rng, 64, 16.0)
    offs = np.zeros((1, 2), np.int32)
    y = datagen.simulate(rng, x, d, offs, 1e5)
    w = datagen.Workload("single", x, d, offs, y, 1e5, 9)
    _check_iteration(w, 3)


def test_nonsquare_ragged_uncovered():
    """Non-square image whose sides are not tile multiples, with an uncovered border."""
    rng = np.random.Generator(np.random.PCG64(10))
    x = datagen.make_object(rng, 150, 230)
    d = datagen.make_probe(rng, 32, 8.0)
    offs = np.array([(r, c) for r in range(5, 150 - 32 - 4, 9) for c in range(3, 230 - 32 - 6, 11)],
                    dtype=np.int32)
    y = datagen.simulate(rng, x, d, offs, 1e5)
    w = datagen.Workload("ragged", x, d, offs, y, 1e5, 10)
    g, o = _check_iteration(w, 2)
    from oracle import pmace_oracle as orc
    lam = orc.weight_image(w.probe, w.offsets, w.x.shape, 1.25)
    assert (lam == 0).any()
    assert np.all(g["x_hat"][lam == 0] == 0)


def test_zero_probe_pixels():
    """Where |d| vanishes the agent returns its input at that pixel."""
    w = datagen.make_workload("small", seed=11)
    probe = w.probe.copy()
    probe[0, :5] = 0
    probe[31, 31] = 0
    y = datagen.simulate(np.random.Generator(np.random.PCG64(11)), w.x, probe, w.offsets, 1e5)
    x0 = random_start(w)
    g = run_gpu(w, 2, 0.5, 0.5, probe=probe, y=y, init=x0)
    o = run_oracle(w, 2, 0.5, 0.5, probe=probe, y=y, x0=x0)
    assert rel_l2(g["x_hat"], o["x_hat"]) < TOL_ITER
    assert rel_l2(g["v"], o["v"]) < TOL_ITER


def test_constant_start_small():
    """The default energy-matched constant start on the 32 x 32 probe."""
    w = datagen.make_workload("small", seed=12)
    g = run_gpu(w, 2, 0.5, 0.5)
    o = run_oracle(w, 2, 0.5, 0.5)
    assert rel_l2(g["x_hat"], o["x_hat"]) < TOL_ITER


def test_rejects_negative_amplitudes_on_device():
    import torch

    from paper_2111_14240_gb300 import pmace as pm
    w = datagen.make_workload("small", seed=13)
    y = w.y.astype(np.float32)
    y[5, 3, 4] = -1.0
    with pytest.raises(pm.PmaceError) as e:
        pm.Reconstruction(w.probe, w.offsets, torch.from_numpy(y).cuda(), w.x.shape)
    assert e.value.status == pm.PMACE_ERR_INVALID_ARG


@pytest.mark.parametrize("cfg,variant", [("small", 4), ("mid64", 4), ("mid128", 4), ("mid128", 5), ("p256", 4)])
def test_forward_transform_stage_matches_fft(cfg, variant):
    """The agent sweep's forward 2-D DFT on its own (the exchange plans' row
    and column stages, before the magnitude replacement, Section III-A)
    against numpy's orthonormal FFT of d v_j for every window, the
    digit-reversed order undone: from a start image the first iteration's
    agent input is v_j = P_j x0."""
    import torch

    from paper_2111_14240_gb300 import pmace as pm
    from tests.gpu_helpers import plan_env
    spec = {"small": "small", "mid64": dict(MID64, name="mid64"), "mid128": dict(MID128, name="mid128"),
            "p256": "p256"}[cfg]
    w = datagen.make_workload(spec, seed=41)
    _, _, probe32, y32 = rounded_inputs(w)
    x0 = random_start(w)
    with plan_env(variant):
        rec = pm.Reconstruction(probe32, w.offsets, y32, w.x.shape, init=x0)
    try:
        assert rec.plan()["variant"] == variant
        out = torch.empty((w.J, w.np_, w.np_, 2), dtype=torch.float32, device="cuda")
        pm.pmace_debug_spectra(rec.h, 0.5, 0.5, out)
        got = torch.view_as_complex(out).cpu().numpy().astype(np.complex128) / w.np_
    finally:
        rec.close()
    v = np.stack([x0[r:r + w.np_, c:c + w.np_] for r, c in w.offsets]).astype(np.complex128)
    ref = np.fft.fft2(probe32.astype(np.complex128)[None] * v, norm="ortho")
    e = rel_l2(got, ref)
    print(f"{cfg} variant {variant}: forward transform rel-L2 {e:.2e}")
    assert e < 2e-6
