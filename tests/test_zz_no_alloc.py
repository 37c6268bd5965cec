"""The allocation-free entry point pmace_amplitude_energy_noalloc.

It serves callers that cannot allocate device memory (their memory is owned
by another allocator, or they must avoid the device-wide synchronisation of
cudaMalloc/cudaFree).  It computes the same total energy sum_j ||y_j||^2 that
pmace_create uses for its energy-matched starting constant
c = sqrt(sum_j ||y_j||^2 / (J ||d||^2)); the test recovers c from both routes
and compares them, on two calls in a row (the calls share one fixed scratch
array).  Collected last on purpose, and self-contained so that it also runs
alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2111_14240_gb300 import datagen
from tests.gpu_helpers import TOL_ITER, rounded_inputs

pytestmark = pytest.mark.gpu


def _existing_constant(pm, w, amps, fmt, scales):
    """Start value c from the existing path: create a job with the default
    start and read a patch of the initial stack (every value equals c)."""
    _, _, probe32, _ = rounded_inputs(w)
    rec = pm.Reconstruction(probe32, w.offsets, amps, w.x.shape, amp_format=fmt, scales=scales)
    try:
        v = rec.patches()[0].cpu().numpy()
    finally:
        rec.close()
    assert np.all(v == v.flat[0])
    return float(v.flat[0].real)


@pytest.mark.parametrize("f16", [False, True])
def test_noalloc_energy_matches_create_start_constant(f16):
    import torch

    from paper_2111_14240_gb300 import build
    build.build()
    from paper_2111_14240_gb300 import pmace as pm

    torch.cuda.init()
    w = datagen.make_workload("small", seed=31)
    _, _, probe32, y32 = rounded_inputs(w)
    J, n = w.J, w.np_
    if f16:
        codes, scales = datagen.quantize_amplitudes_f16(y32.astype(np.float64))
        amps = torch.from_numpy(codes).cuda()
        sc = torch.from_numpy(scales).cuda()
        fmt = pm.PMACE_AMP_F16_SCALED
        # the device forms code * scale in FP32, as pmace_create does
        y_host = (codes.astype(np.float32) * scales[:, None, None]).astype(np.float64)
    else:
        amps = torch.from_numpy(y32).cuda()
        sc = None
        fmt = pm.PMACE_AMP_F32
        y_host = y32.astype(np.float64)
    c_existing = _existing_constant(pm, w, amps, fmt, sc)
    d2 = float(np.sum(np.abs(probe32.astype(np.complex128)) ** 2))
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(-1.0)
        pm.pmace_amplitude_energy_noalloc(amps, J, n, out, amp_format=fmt, scales=sc)
        torch.cuda.synchronize()
        energy = float(out.item())
        c_new = np.sqrt(energy / (J * d2))
        assert abs(c_new - c_existing) <= TOL_ITER * c_existing, (c_new, c_existing)
        assert abs(energy - np.sum(y_host ** 2)) <= 1e-12 * energy


def test_noalloc_rejects_too_many_windows():
    import torch

    from paper_2111_14240_gb300 import pmace as pm
    amps = torch.zeros(4, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = pm._lib.pmace_amplitude_energy_noalloc(ctypes.c_void_p(amps.data_ptr()), pm.PMACE_AMP_F32,
                                                None, 65537, 1, ctypes.c_void_p(out.data_ptr()), None)
    assert st == pm.PMACE_ERR_INVALID_ARG
    assert "65536" in pm.pmace_last_error(None)
