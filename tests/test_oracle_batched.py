"""The batched CPU baseline (all host cores) against the literal oracle: the
same Algorithm 1 iterates, to rounding (CPU only)."""
import numpy as np

from oracle import pmace_batched, pmace_oracle
from paper_2111_14240_gb300 import datagen


def test_batched_oracle_matches_literal_oracle():
    w = datagen.make_workload("small", seed=4)
    kw = dict(alpha=0.6, rho=0.45, kappa=1.25, n_iter=3)
    a = pmace_oracle.pmace(w.y, w.probe, w.offsets, w.x.shape, **kw)
    b = pmace_batched.pmace(w.y, w.probe, w.offsets, w.x.shape, workers=2, **kw)
    for k in ("v", "w", "z", "xbar", "x_hat"):
        assert np.linalg.norm(b[k] - a[k]) <= 1e-12 * np.linalg.norm(a[k]), k


def test_batched_agent_absent_probe_pixels():
    """The absent-probe reading (|d| <= 1e-30 max|d| returns the input)
    holds in the batched agent as in the literal one."""
    rng = np.random.Generator(np.random.PCG64(3))
    d = datagen.make_probe(rng, 8, 2.0)
    d[0, 0] = 0.0
    v = rng.standard_normal((3, 8, 8)) + 1j * rng.standard_normal((3, 8, 8))
    y = np.abs(rng.standard_normal((3, 8, 8))) + 0.1
    got = pmace_batched.agents_batched(v, y, d, 0.4, workers=1)
    ref = pmace_oracle.agents(v, y, d, 0.4)
    assert np.array_equal(got[:, 0, 0], v[:, 0, 0])
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
