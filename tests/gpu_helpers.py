"""Shared helpers for the GPU parity tests: run the CUDA path through the C
ABI binding and the FP64 oracle on the same (FP32-rounded) inputs."""
from __future__ import annotations

import contextlib
import os

import numpy as np

from paper_2111_14240_gb300 import datagen

# One full PMACE iteration in FP32 must match the FP64 oracle to this
# relative L2 error, and the end-to-end NRMSE must agree within 1 %.
TOL_ITER = 1e-5
TOL_NRMSE_REL = 0.01


def rel_l2(a, b) -> float:
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rounded_inputs(w: datagen.Workload):
    """The inputs exactly as the GPU sees them (complex64 probe, float32 y),
    returned in float64 for the oracle, plus the float32 arrays for the GPU."""
    probe32 = w.probe.astype(np.complex64)
    y32 = w.y.astype(np.float32)
    return probe32.astype(np.complex128), y32.astype(np.float64), probe32, y32


@contextlib.contextmanager
def plan_env(variant):
    """Select agent kernel variant `variant` (an index of the per-probe-size
    plan table) for jobs created inside the block."""
    old = os.environ.get("PMACE_AGENT_PLAN")
    if variant is not None:
        os.environ["PMACE_AGENT_PLAN"] = str(variant)
    try:
        yield
    finally:
        if old is None:
            os.environ.pop("PMACE_AGENT_PLAN", None)
        else:
            os.environ["PMACE_AGENT_PLAN"] = old


def random_start(w: datagen.Workload, seed: int = 5) -> np.ndarray:
    """A well-conditioned start image (random amplitude and phase per pixel),
    already rounded to complex64.  From the constant start the spectrum of
    d * c is mostly below FP32 resolution, so phases there are undetermined
    in any FP32 implementation; a random start keeps every coefficient
    resolvable and isolates the arithmetic of one iteration."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x0 = rng.uniform(0.5, 1.0, w.x.shape) * np.exp(1j * rng.uniform(0, 2 * np.pi, w.x.shape))
    return x0.astype(np.complex64)


def run_gpu(w: datagen.Workload, iters: int, alpha: float, rho: float = 0.5, *, kappa=1.25,
            variant=None, f16=False, init=None, probe=None, y=None, want_patches=True,
            state=None):
    """Run the CUDA path; returns dict(x_hat, v, r_fp, r_data, plan).
    `state` = (q, xbar, iterations, rho_pending) loads a saved Algorithm 1
    state (complex arrays) before iterating."""
    import torch

    from paper_2111_14240_gb300 import pmace as pm

    _, _, probe32, y32 = rounded_inputs(w)
    if probe is not None:
        probe32 = probe.astype(np.complex64)
    if y is not None:
        y32 = y.astype(np.float32)
    with plan_env(variant):
        if f16:
            codes, scales = datagen.quantize_amplitudes_f16(y32.astype(np.float64))
            rec = pm.Reconstruction(probe32, w.offsets, torch.from_numpy(codes).cuda(), w.x.shape,
                                    kappa=kappa, amp_format=pm.PMACE_AMP_F16_SCALED,
                                    scales=torch.from_numpy(scales).cuda(), init=init)
        else:
            rec = pm.Reconstruction(probe32, w.offsets, y32, w.x.shape, kappa=kappa, init=init)
    try:
        plan = rec.plan()
        if state is not None:
            import torch
            q, xb, n_done, rho_p = state
            qt = torch.view_as_real(torch.from_numpy(q.astype(np.complex64))).contiguous().cuda()
            xt = torch.view_as_real(torch.from_numpy(xb.astype(np.complex64))).contiguous().cuda()
            pm.pmace_set_state(rec.h, qt, xt, pm.pmace_state_info(int(n_done), float(rho_p), 0))
        if iters:
            rec.iterate(iters, alpha, rho)
        out = dict(x_hat=rec.image().cpu().numpy().astype(np.complex128), plan=plan)
        if want_patches:
            out["v"] = rec.patches().cpu().numpy().astype(np.complex128)
        if iters:
            out["r_fp"], out["r_data"] = rec.residual()
        torch.cuda.synchronize()
        return out
    finally:
        rec.close()


def run_oracle(w: datagen.Workload, iters: int, alpha: float, rho: float = 0.5, *, kappa=1.25,
               f16=False, x0=None, probe=None, y=None, v0=None, z_prev=None):
    from oracle import pmace_oracle as orc

    probe64, y64, _, _ = rounded_inputs(w)
    if probe is not None:
        probe64 = probe.astype(np.complex64).astype(np.complex128)
    if y is not None:
        y64 = y.astype(np.float32).astype(np.float64)
    if f16:
        codes, scales = datagen.quantize_amplitudes_f16(y64)
        y64 = datagen.dequantize_f16(codes, scales)
    if x0 is not None:
        x0 = x0.astype(np.complex64).astype(np.complex128)
    return orc.pmace(y64, probe64, w.offsets, w.x.shape, alpha=alpha, rho=rho, kappa=kappa,
                     n_iter=iters, x0=x0, v0=v0, z_prev=z_prev)


def fused_state(res: dict, rho: float):
    """Algorithm 1 state after an oracle run in the library's checkpoint form:
    q = v - 2 rho z (so that v = q + 2 rho P xbar) and xbar."""
    return res["v"] - 2.0 * rho * res["z"], res["xbar"]
