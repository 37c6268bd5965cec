"""FP16 amplitudes with a per-pattern FP32 scale against FP32 amplitudes, end
to end: the geometry of the 2048 x 2048 / 128 x 128 workload (step 16 px,
+-2 px jitter) on a 30 x 30 scan, measurements made by the GPU simulator at
Poisson peaks 1e4 and 1e6, 200 iterations on each path.  The FP16 path's
reconstruction error must be within 1 % of the FP32 path's."""
import numpy as np
import pytest

from paper_2111_14240_gb300 import datagen
from tests.gpu_helpers import TOL_NRMSE_REL

pytestmark = pytest.mark.gpu


def _nrmse(x_hat, x, mask):
    a, b = x_hat[mask].astype(np.complex128), x[mask]
    theta = np.angle(np.vdot(b, a))
    return float(np.linalg.norm(a - np.exp(1j * theta) * b) / np.linalg.norm(b))


@pytest.mark.parametrize("peak", [1e4, 1e6])
def test_f16_amplitudes_reconstruct_as_well_as_f32(peak):
    import torch

    from paper_2111_14240_gb300 import build
    from paper_2111_14240_gb300 import pmace as pm
    build.build()
    rng = np.random.Generator(np.random.PCG64(11))
    n_obj, n_p, n_scan = 600, 128, 30
    x = datagen.make_object(rng, n_obj, n_obj)
    probe = datagen.make_probe(rng, n_p, 32.0)
    offs = datagen.make_offsets(rng, n_obj, n_p, n_scan, 16, 2)
    y = pm.simulate(x, probe, offs, peak=peak, seed=5)
    codes, scales = datagen.quantize_amplitudes_f16(y.astype(np.float64))
    mask = np.zeros(x.shape, bool)
    for r, c in offs:
        mask[r:r + n_p, c:c + n_p] = True
    err = {}
    for f16 in (False, True):
        if f16:
            rec = pm.Reconstruction(probe.astype(np.complex64), offs, torch.from_numpy(codes).cuda(), x.shape,
                                    amp_format=pm.PMACE_AMP_F16_SCALED, scales=torch.from_numpy(scales).cuda())
        else:
            rec = pm.Reconstruction(probe.astype(np.complex64), offs, y, x.shape)
        try:
            rec.iterate(200, 0.5, 0.5)
            err[f16] = _nrmse(rec.image().cpu().numpy(), x, mask)
        finally:
            rec.close()
    print(f"peak {peak:g}: NRMSE FP32 {err[False]:.5f} FP16 {err[True]:.5f}")
    assert abs(err[True] - err[False]) <= TOL_NRMSE_REL * err[False]
