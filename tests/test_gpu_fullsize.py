"""Full-size workloads checked on sampled windows.

For the 2048 x 2048 / 128 x 128 / 14641-window workload (FP32 and FP16
amplitudes) and the 8192 x 8192 / 64009-window workload the oracle cannot
run a whole iteration in seconds, but one window's result after one
iteration depends only on the windows that overlap it: the oracle computes
the agent outputs of those windows, the consensus image on the sampled
window's pixels (the weight image there only involves the same windows) and
the Mann update, and compares with the GPU's stack for that window.
"""
import os

import numpy as np
import pytest

from oracle import pmace_oracle as orc
from paper_2111_14240_gb300 import datagen
from tests.gpu_helpers import TOL_ITER, random_start, rel_l2, rounded_inputs

pytestmark = pytest.mark.gpu


def _neighbours(offs, j, n_p):
    r, c = offs[j]
    return np.where((np.abs(offs[:, 0] - r) < n_p) & (np.abs(offs[:, 1] - c) < n_p))[0]


def _oracle_window_after_one_iteration(w, y64, probe64, x0, j, alpha, rho, kappa=1.25):
    """v_j after one Algorithm 1 iteration from the start image x0."""
    n_p = probe64.shape[0]
    nb = _neighbours(w.offsets, j, n_p)
    offs = w.offsets[nb]
    v0 = orc.redistribute(x0, offs, n_p)
    wstack = orc.agents(v0, y64[nb], probe64, alpha)
    lam_inv = orc.inverse_weights(orc.weight_image(probe64, offs, x0.shape, kappa))
    xbar = orc.consensus_image(2.0 * wstack - v0, probe64, offs, lam_inv, kappa)
    k = int(np.where(nb == j)[0][0])
    z = orc.extract(xbar, offs[k], n_p)
    return v0[k] + 2.0 * rho * (z - wstack[k])


def run_boundary_samples(J, wpc, n_scan):
    """Windows to sample: the first and last, both sides of the first cluster
    run's end, of a run boundary near the middle and of the last run's
    start (a cluster of the agent sweep processes wpc consecutive windows),
    both sides of the first raster row's end, and an interior window off
    every boundary."""
    mid = (J // 2 // wpc) * wpc
    last = ((J - 1) // wpc) * wpc
    s = {0, wpc - 1, wpc, mid - 1, mid, last - 1, last, n_scan - 1, n_scan, J // 2 + 17, J - 1}
    return sorted(j for j in s if 0 <= j < J)


def _check(w, f16, samples, alpha=0.5, rho=0.5):
    import torch

    from paper_2111_14240_gb300 import pmace as pm
    probe64, y64, probe32, y32 = rounded_inputs(w)
    x0 = random_start(w).astype(np.complex64)
    if f16:
        codes, scales = datagen.quantize_amplitudes_f16(y64)
        y64 = datagen.dequantize_f16(codes, scales)
        rec = pm.Reconstruction(probe32, w.offsets, torch.from_numpy(codes).cuda(), w.x.shape,
                                amp_format=pm.PMACE_AMP_F16_SCALED,
                                scales=torch.from_numpy(scales).cuda(), init=x0)
    else:
        rec = pm.Reconstruction(probe32, w.offsets, y32, w.x.shape, init=x0)
    try:
        rec.iterate(1, alpha, rho)
        v = rec.patches()
        plan = rec.plan()
        if callable(samples):
            samples = samples(w.J, plan["windows_per_cluster"])
        got = {j: v[j].cpu().numpy().astype(np.complex128) for j in samples}
    finally:
        rec.close()
        del v
        torch.cuda.empty_cache()
    x0d = x0.astype(np.complex128)
    for j in samples:
        ref = _oracle_window_after_one_iteration(w, y64, probe64, x0d, j, alpha, rho)
        e_w = rel_l2(got[j] * np.abs(probe64), ref * np.abs(probe64))
        e = rel_l2(got[j], ref)
        print(f"{w.name} J={w.J} f16={f16} plan={plan} window {j}: |d|v {e_w:.2e} v {e:.2e}")
        assert e_w < TOL_ITER and e < TOL_ITER


@pytest.fixture(scope="module")
def p128():
    return datagen.make_workload("p128", seed=1)


@pytest.mark.parametrize("f16", [False, True])
def test_p128_full_size_sampled(p128, f16):
    n_scan = datagen.CONFIGS["p128"]["n_scan"]
    _check(p128, f16, samples=lambda J, wpc: run_boundary_samples(J, wpc, n_scan))


@pytest.mark.skipif(os.environ.get("PMACE_SKIP_LARGE") == "1", reason="large workload skipped on request")
def test_large_full_size_sampled_f16():
    """8192 x 8192 object, 64009 windows of 128 x 128, FP16 amplitudes."""
    w = datagen.make_workload("large", seed=1)
    n_scan = datagen.CONFIGS["large"]["n_scan"]
    _check(w, True, samples=lambda J, wpc: run_boundary_samples(J, wpc, n_scan))
