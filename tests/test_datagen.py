"""Host-side checks of the seeded workload generator (CPU only)."""
import numpy as np

from paper_2111_14240_gb300 import datagen


def test_small_workload_shapes_and_ranges():
    w = datagen.make_workload("small", seed=1)
    assert w.x.shape == (128, 128) and w.probe.shape == (32, 32)
    assert w.offsets.shape == (169, 2) and w.offsets.dtype == np.int32
    assert w.offsets.min() >= 0 and w.offsets.max() <= 128 - 32
    amp, ph = np.abs(w.x), np.angle(w.x)
    assert abs(amp.min() - 0.6) < 1e-12 and abs(amp.max() - 1.0) < 1e-12
    assert abs(ph.min()) < 1e-12 and abs(ph.max() - np.pi / 2) < 1e-12
    assert abs(np.abs(w.probe).max() - np.exp(-0.5 * 0.5 / 64)) < 1e-3
    assert w.y.shape == (169, 32, 32) and np.all(w.y >= 0)


def test_seeded_and_reproducible():
    a = datagen.make_workload("small", seed=2)
    b = datagen.make_workload("small", seed=2)
    c = datagen.make_workload("small", seed=3)
    assert np.array_equal(a.y, b.y) and np.array_equal(a.offsets, b.offsets)
    assert not np.array_equal(a.y, c.y)


def test_noiseless_matches_forward_model():
    w = datagen.make_workload("small", seed=1, noiseless=True)
    j = 17
    r, c = w.offsets[j]
    ref = np.abs(np.fft.fft2(w.probe * w.x[r:r + 32, c:c + 32], norm="ortho"))
    assert np.max(np.abs(w.y[j] - ref)) < 1e-12


def test_poisson_scaling_peak():
    """Per-pattern scaling: the brightest pixel of each pattern has ~peak counts."""
    w = datagen.make_workload("small", seed=1)
    wn = datagen.make_workload("small", seed=1, noiseless=True)
    m = (wn.y.reshape(169, -1) ** 2).max(axis=1)
    counts = (w.y.reshape(169, -1) ** 2) * (1e5 / m[:, None])
    assert np.allclose(counts, np.round(counts), atol=1e-6 * 1e5)
    rel = np.abs(counts.max(axis=1) - 1e5) / 1e5
    assert np.all(rel < 0.02)


def test_f16_quantisation():
    w = datagen.make_workload("small", seed=1)
    codes, s = datagen.quantize_amplitudes_f16(w.y)
    assert codes.dtype == np.float16 and s.dtype == np.float32
    assert codes.max() <= 1.0
    yq = datagen.dequantize_f16(codes, s)
    assert np.max(np.abs(yq - w.y) / s[:, None, None]) < 2 ** -11


def test_raster_geometry_p256():
    rng = np.random.Generator(np.random.PCG64(0))
    offs = datagen.make_offsets(rng, 600, 256, 18, 20, 0)
    assert offs[0, 0] == 2 and offs[-1, 0] == 2 + 17 * 20
