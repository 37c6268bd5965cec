"""FP64 CPU oracle of the data simulator (Section II forward model plus the
Section IV photon scaling), for arXiv 2111.14240.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or runs
this file: only the tests do.  It shares no code with the CUDA path.

* forward model (Section II): the intensity of window j is
  I_j = |F D P_j x|^2 with F the 2-D orthonormal DFT (DC at index 0);
* photon scaling (Section IV): with M_j = max over the window of I_j and the
  peak count r, the measured amplitude is y_j = sqrt(Pois(I_j r / M_j)) *
  sqrt(M_j / r) (y_j = sqrt(I_j) without noise; y_j = 0 where M_j = 0);
* the random numbers come from the counter-based generator Philox4x32-10
  (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
  SC 2011), written here from its published definition; draw n of pixel p
  of window j uses counter (p, j, n, 0x504d4143) and key (seed low word,
  seed high word), and two 32-bit words (a, b) make one double
  ((a >> 5) 2^26 + (b >> 6)) / 2^53 in [0, 1), two doubles per call;
* Poisson sampling: Knuth's multiplication method for lambda < 10 and the
  transformed rejection method with squeeze (PTRS) of W. Hoermann, "The
  transformed rejection method for generating Poisson random variables",
  Insurance: Mathematics and Economics 12 (1993), for lambda >= 10, both in
  FP64.

Pins (tests/test_simulate_oracle.py): the generator against its published
known-answer values, uniformity and independence of the doubles, Poisson
means and variances against lambda, the noiseless forward model against
Parseval and a closed form, and the noisy amplitudes' scaling.
"""
from __future__ import annotations

import numpy as np
from scipy.special import gammaln

from oracle.pmace_oracle import extract, fft2o

MASK = np.uint64(0xFFFFFFFF)
PHILOX_M0, PHILOX_M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
PHILOX_W0, PHILOX_W1 = np.uint64(0x9E3779B9), np.uint64(0xBB67AE85)
STREAM_TAG = 0x504D4143


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on arrays of 32-bit words (held in uint64).

    A round multiplies word 0 by M0 and word 2 by M1 (64-bit products split
    into high and low halves) and outputs (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2),
    hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key is bumped by the Weyl constants
    (W0, W1) before every round after the first.
    """
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & MASK for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & MASK
    k1 = np.asarray(k1, dtype=np.uint64) & MASK
    for r in range(10):
        if r > 0:
            k0 = (k0 + PHILOX_W0) & MASK
            k1 = (k1 + PHILOX_W1) & MASK
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        c0, c1, c2, c3 = ((p1 >> np.uint64(32)) ^ c1 ^ k0, p1 & MASK,
                          (p0 >> np.uint64(32)) ^ c3 ^ k1, p0 & MASK)
    return c0, c1, c2, c3


def words_to_double(a, b):
    """53-bit double in [0, 1) from two 32-bit words."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    return ((a >> np.uint64(5)).astype(np.float64) * 67108864.0
            + (b >> np.uint64(6)).astype(np.float64)) / 9007199254740992.0


class Streams:
    """Per-pixel uniform streams: one stream per (window j, pixel p)."""

    def __init__(self, seed: int, j, p):
        self.j = np.asarray(j, dtype=np.uint64)
        self.p = np.asarray(p, dtype=np.uint64)
        self.k0 = np.uint64(seed & 0xFFFFFFFF)
        self.k1 = np.uint64((seed >> 32) & 0xFFFFFFFF)
        self.n = np.zeros(self.p.shape, dtype=np.uint64)      # Philox calls made
        self.spare = np.full(self.p.shape, np.nan)             # second double of the last call

    def next(self, active):
        """The next uniform of every active stream (in stream order)."""
        out = np.empty(int(np.count_nonzero(active)))
        idx = np.nonzero(active)[0]
        have = ~np.isnan(self.spare[idx])
        out[have] = self.spare[idx[have]]
        self.spare[idx[have]] = np.nan
        need = idx[~have]
        if need.size:
            w = philox4x32_10(self.p[need], self.j[need], self.n[need], STREAM_TAG, self.k0, self.k1)
            self.n[need] += np.uint64(1)
            out[~have] = words_to_double(w[0], w[1])
            self.spare[need] = words_to_double(w[2], w[3])
        return out


def poisson(lam: np.ndarray, streams: Streams) -> np.ndarray:
    """Poisson samples for every lambda (FP64), one stream each."""
    lam = np.asarray(lam, dtype=np.float64)
    k = np.zeros(lam.shape, dtype=np.int64)
    # Knuth: the count of uniforms whose running product stays above exp(-lambda)
    small = (lam > 0) & (lam < 10)
    lim = np.exp(-lam)
    prod = np.ones(lam.shape)
    active = small.copy()
    for _ in range(4096):   # the same bound as the CUDA sampler (never reached)
        if not active.any():
            break
        prod[active] *= streams.next(active)
        go = active & (prod > lim)
        k[go] += 1
        active = go
    # PTRS
    big = lam >= 10
    slam = np.sqrt(lam)
    loglam = np.log(np.where(big, lam, 1.0))
    b = 0.931 + 2.53 * slam
    a = -0.059 + 0.02483 * b
    invalpha = 1.1239 + 1.1328 / (b - 3.4)
    vr = 0.9277 - 3.6224 / (b - 2.0)
    active = big.copy()
    while active.any():
        idx = np.nonzero(active)[0]
        u = streams.next(active) - 0.5
        v = streams.next(active)
        us = 0.5 - np.abs(u)
        kk = np.floor((2.0 * a[idx] / us + b[idx]) * u + lam[idx] + 0.43)
        acc = (us >= 0.07) & (v <= vr[idx])
        rej = ~acc & ((kk < 0) | ((us < 0.013) & (v > us)))
        test = ~acc & ~rej
        if test.any():
            t = idx[test]
            lhs = np.log(v[test]) + np.log(invalpha[t]) - np.log(a[t] / (us[test] * us[test]) + b[t])
            rhs = -lam[t] + kk[test] * loglam[t] - gammaln(kk[test] + 1.0)
            acc[np.nonzero(test)[0]] = lhs <= rhs
        k[idx[acc]] = kk[acc].astype(np.int64)
        active[idx[acc]] = False
    return k


def intensities(x: np.ndarray, probe: np.ndarray, offsets: np.ndarray) -> np.ndarray:
    """I_j = |F D P_j x|^2 for every window (Section II), FP64."""
    n_p = probe.shape[0]
    return np.stack([np.abs(fft2o(probe * extract(x, o, n_p))) ** 2 for o in offsets])


def noisy_amplitudes(inten: np.ndarray, peak: float, seed: int) -> np.ndarray:
    """Section IV photon scaling of given intensities (J, Np, Np), FP64:
    y = sqrt(Pois(I r / M)) * sqrt(M / r) with M the window maximum."""
    J, n1, n2 = inten.shape
    flat = inten.reshape(J, -1).astype(np.float64)
    m = flat.max(axis=1)
    scale = np.where(m > 0, peak / np.where(m > 0, m, 1.0), 0.0)
    lam = flat * scale[:, None]
    jj, pp = np.meshgrid(np.arange(J), np.arange(n1 * n2), indexing="ij")
    counts = poisson(lam.ravel(), Streams(seed, jj.ravel(), pp.ravel())).reshape(J, -1)
    y = np.sqrt(counts.astype(np.float64)) * np.sqrt(m / peak)[:, None]
    return y.reshape(J, n1, n2)


def simulate(x, probe, offsets, peak: float | None, seed: int = 0) -> np.ndarray:
    """Measured amplitudes y_j (J, Np, Np): sqrt(I_j) without noise, else the
    photon-scaled Poisson draw."""
    inten = intensities(x, probe, offsets)
    if peak is None or peak <= 0:
        return np.sqrt(inten)
    return noisy_amplitudes(inten, peak, seed)
