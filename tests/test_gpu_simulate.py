"""The GPU data simulator (pmace_simulate, pmace_photon_noise) against the
simulator oracle (oracle/simulate_oracle.py), through the C ABI.

* The noiseless forward model |F D P_j x| matches the FP64 oracle within the
  parity bound on every probe size, the full 324-window workload included.
* The photon scaling, given the same float32 intensities, matches the
  oracle bit for bit: the same Philox4x32-10 streams and the same Poisson
  algorithms, every step in FP64.
* The whole noisy pipeline: the GPU's FP32 intensities differ from the
  oracle's FP64 ones by rounding, so a count can differ where a draw falls
  at a decision boundary; almost all agree exactly and the rest by a count.
"""
import numpy as np
import pytest

from oracle import simulate_oracle as so
from paper_2111_14240_gb300 import datagen
from tests.gpu_helpers import TOL_ITER, rel_l2

pytestmark = pytest.mark.gpu

MID64 = dict(n_obj=200, n_p=64, probe_sigma=16.0, n_scan=9, step=16, jitter=2, peak=1e5, name="mid64")
MID128 = dict(n_obj=400, n_p=128, probe_sigma=32.0, n_scan=9, step=32, jitter=2, peak=1e5, name="mid128")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2111_14240_gb300 import build
    build.build()


def _inputs(cfg, seed):
    w = datagen.make_workload(cfg, seed=seed)
    x = w.x.astype(np.complex64)
    d = w.probe.astype(np.complex64)
    return w, x, d


@pytest.mark.parametrize("cfg", ["small", MID64, MID128, "p256"], ids=["np32", "np64", "np128", "np256"])
def test_noiseless_forward_model(cfg):
    from paper_2111_14240_gb300 import pmace as pm
    w, x, d = _inputs(cfg, 21)
    got = pm.simulate(x, d, w.offsets)
    ref = np.sqrt(so.intensities(x.astype(np.complex128), d.astype(np.complex128), w.offsets))
    e = rel_l2(got.astype(np.float64), ref)
    print(f"np={w.np_} J={w.J}: noiseless amplitudes rel-L2 {e:.2e}")
    assert e < TOL_ITER


@pytest.mark.parametrize("peak", [1e3, 1e5])
def test_photon_noise_is_bit_exact(peak):
    """Same float32 intensities in: every count, hence every amplitude, equal."""
    from paper_2111_14240_gb300 import pmace as pm
    w, x, d = _inputs("small", 22)
    inten = so.intensities(x.astype(np.complex128), d.astype(np.complex128), w.offsets).astype(np.float32)
    inten[3] = 0.0                                   # a window with nothing measured
    got = pm.photon_noise(inten, peak, seed=0x1234_5678_9ABC)
    ref = so.noisy_amplitudes(inten.astype(np.float64), peak, seed=0x1234_5678_9ABC).astype(np.float32)
    lam = inten.reshape(w.J, -1) * (peak / np.maximum(inten.reshape(w.J, -1).max(axis=1, keepdims=True), 1e-30))
    print(f"peak {peak}: lambda < 10 for {np.mean(lam < 10):.2%} of pixels, max {lam.max():.3g}")
    assert np.all(got[3] == 0)
    assert np.array_equal(got, ref)
    # the same seed again: the same draw; another seed: another draw
    assert np.array_equal(pm.photon_noise(inten, peak, seed=0x1234_5678_9ABC), got)
    assert not np.array_equal(pm.photon_noise(inten, peak, seed=7), got)


def test_noisy_pipeline_against_oracle():
    from paper_2111_14240_gb300 import pmace as pm
    w, x, d = _inputs(MID64, 23)
    peak = 1e4
    got = pm.simulate(x, d, w.offsets, peak=peak, seed=99).astype(np.float64)
    ref = so.simulate(x.astype(np.complex128), d.astype(np.complex128), w.offsets, peak, seed=99)
    inten = so.intensities(x.astype(np.complex128), d.astype(np.complex128), w.offsets)
    m = inten.reshape(w.J, -1).max(axis=1)[:, None, None]
    cg = np.rint(got ** 2 * peak / m)
    cr = np.rint(ref ** 2 * peak / m)
    same = np.mean(cg == cr)
    print(f"counts equal for {same:.5%} of pixels; largest difference {np.abs(cg - cr).max()}")
    assert same > 0.999 and np.abs(cg - cr).max() <= 2
    # and the noise has the forward model's mean: E[y^2] = I
    assert abs(np.sum(got ** 2) / np.sum(inten) - 1) < 1e-2


def test_simulated_data_reconstructs():
    """Amplitudes made on the GPU feed pmace_create directly (same layout)."""
    from paper_2111_14240_gb300 import pmace as pm
    w, x, d = _inputs("small", 24)
    y = pm.simulate(x, d, w.offsets)
    rec = pm.Reconstruction(d, w.offsets, y, w.x.shape)
    try:
        rec.iterate(30, 0.5, 0.5)
        r_fp, r_data = rec.residual()
    finally:
        rec.close()
    assert r_data < 0.05


def test_simulator_rejects_bad_input():
    from paper_2111_14240_gb300 import pmace as pm
    w, x, d = _inputs("small", 25)
    with pytest.raises(pm.PmaceError):
        pm.simulate(x, d[:24, :24], w.offsets[:4] * 0)      # probe size 24 is unsupported
    bad = w.offsets.copy()
    bad[0, 0] = x.shape[0]                                  # window past the edge
    with pytest.raises(pm.PmaceError):
        pm.simulate(x, d, bad)
