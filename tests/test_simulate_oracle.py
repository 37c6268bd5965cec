"""Pins of the simulator oracle (oracle/simulate_oracle.py) against what the
generator's definition, probability theory and the forward model fix."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import simulate_oracle as so

KAT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    for line in open(KAT):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        got = so.philox4x32_10(*v[:6])
        assert [int(g) for g in got] == v[6:]


def test_uniform_doubles_are_uniform_and_independent():
    n = 200000
    s = so.Streams(12345, np.zeros(n, np.int64), np.arange(n))
    u = s.next(np.ones(n, bool))
    w = s.next(np.ones(n, bool))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 0.002
    assert abs(np.corrcoef(u, w)[0, 1]) < 5 / np.sqrt(n)
    # the same (seed, window, pixel) gives the same stream; another seed another
    assert np.array_equal(so.Streams(12345, np.zeros(8, np.int64), np.arange(8)).next(np.ones(8, bool)), u[:8])
    assert not np.array_equal(so.Streams(12346, np.zeros(8, np.int64), np.arange(8)).next(np.ones(8, bool)), u[:8])


@pytest.mark.parametrize("lam", [0.7, 3.0, 9.5, 10.0, 23.0, 400.0, 1.0e5])
def test_poisson_distribution(lam):
    n = 40000
    k = so.poisson(np.full(n, lam), so.Streams(7, np.zeros(n, np.int64), np.arange(n)))
    assert abs(k.mean() - lam) < 5 * np.sqrt(lam / n)
    assert abs(k.var() / lam - 1) < 5 * np.sqrt(2.0 / n) + 0.01
    # chi-square against the Poisson pmf over the central values
    lo, hi = int(stats.poisson.ppf(0.001, lam)), int(stats.poisson.ppf(0.999, lam))
    edges = np.unique(np.linspace(lo, hi + 1, min(40, hi - lo + 2)).astype(int))
    obs = np.histogram(k, bins=edges)[0]
    exp = n * np.diff(stats.poisson.cdf(edges - 1, lam))
    keep = exp > 5
    chi2 = np.sum((obs[keep] - exp[keep]) ** 2 / exp[keep])
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-4


def test_poisson_zero_rate():
    k = so.poisson(np.zeros(16), so.Streams(1, np.zeros(16, np.int64), np.arange(16)))
    assert np.all(k == 0)


def test_intensities_parseval_and_closed_form():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((40, 40)) + 1j * rng.standard_normal((40, 40))
    d = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    offs = np.array([[0, 0], [5, 9], [24, 24]])
    inten = so.intensities(x, d, offs)
    for j, (r, c) in enumerate(offs):
        assert np.isclose(inten[j].sum(), np.sum(np.abs(d * x[r:r + 16, c:c + 16]) ** 2))
    # constant object, constant probe: all energy at DC, |c N|^2
    one = so.intensities(np.full((40, 40), 0.5 + 0.5j), np.ones((16, 16)), offs[:1])[0]
    assert np.isclose(one[0, 0], 16 * 16 * 0.5) and np.allclose(one.ravel()[1:], 0, atol=1e-20)


def test_noisy_amplitudes_scale_and_limits():
    rng = np.random.default_rng(4)
    inten = rng.uniform(0.0, 3.0, (3, 16, 16))
    inten[1] = 0.0
    y = so.noisy_amplitudes(inten, 1e6, seed=9)
    assert np.all(y[1] == 0)                                  # M = 0: nothing measured
    for j in (0, 2):                                          # E[y^2] = I at high counts
        assert np.allclose(y[j] ** 2, inten[j], rtol=0.02, atol=3 * inten[j].max() / 1e3)
    y2 = so.noisy_amplitudes(inten, 1e6, seed=9)
    assert np.array_equal(y, y2)
    # counts are integers: y^2 r / M is integral
    m = inten[0].max()
    assert np.allclose(np.round(y[0] ** 2 * 1e6 / m), y[0] ** 2 * 1e6 / m, atol=1e-6)
