"""Seeded synthetic ptychography workloads.

This module only *draws* inputs: a complex transmittance image x, a probe d,
integer scan offsets and the measured amplitudes y_j.  It holds none of the
reconstruction arithmetic (no agent, no consensus, no Mann step); the
measurements come from the idealised forward model of Section II,
y_j = sqrt(Pois(|F D P_j x|^2)), evaluated with numpy's FFT in float64 and
the per-pattern photon scaling of the noisy-data equation in Section IV.

Recipe (the paper's LANL image and probe are not available, so these stand
in for them):

* object: amplitude drawn U[amp_lo, amp_hi] and phase U[ph_lo, ph_hi] per
  pixel, each smoothed with a periodic Gaussian (sigma px) and then affinely
  rescaled so that its min/max hit the stated bounds;
* probe: Gaussian amplitude (sigma px, peak 1) centred at ((Np-1)/2,(Np-1)/2)
  times a random quadratic phase a*r^2/(Np/2)^2 with a ~ U[0, 2*pi);
* scan: n x n raster with the given step, centred (margin =
  floor((N - (n-1)*step - Np)/2)), each coordinate jittered by an integer
  uniform in [-jitter, jitter] and clamped to [0, N - Np];
* measurements: per pattern j, M_j = max|F D x_j|^2 and
  y_j = sqrt(Pois(|F D x_j|^2 * r_p / M_j)) * sqrt(M_j / r_p), i.e. the
  paper's photon-count model rescaled back to model units so that the
  noiseless limit keeps the ground truth as a fixed point; r_p = None gives
  noiseless y_j = |F D x_j|.

Every draw uses numpy Generator(PCG64(seed)) in a fixed order.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Workload:
    name: str
    x: np.ndarray          # (N1, N2) complex128 ground truth
    probe: np.ndarray      # (Np, Np) complex128
    offsets: np.ndarray    # (J, 2) int32, (row, col) top-left of each window
    y: np.ndarray          # (J, Np, Np) float64 measured amplitudes
    peak: float | None     # photon peak r_p, None when noiseless
    seed: int

    @property
    def np_(self) -> int:
        return self.probe.shape[0]

    @property
    def J(self) -> int:
        return self.offsets.shape[0]


# The workloads: (object side, probe side, probe sigma, raster n, step,
# jitter, photon peak, iterations).
CONFIGS = {
    "small": dict(n_obj=128, n_p=32, probe_sigma=8.0, n_scan=13, step=8,
                  jitter=1, peak=1e5, iters=50),
    "p256": dict(n_obj=600, n_p=256, probe_sigma=48.0, n_scan=18, step=20,
                 jitter=2, peak=1e5, iters=100),
    "p128": dict(n_obj=2048, n_p=128, probe_sigma=32.0, n_scan=121, step=16,
                 jitter=2, peak=1e4, iters=200),
    "large": dict(n_obj=8192, n_p=128, probe_sigma=32.0, n_scan=253, step=32,
                  jitter=3, peak=1e5, iters=100),
}


def _smooth_periodic(a: np.ndarray, sigma: float) -> np.ndarray:
    """Periodic Gaussian blur via the Fourier transform of the kernel."""
    n1, n2 = a.shape
    f1 = np.fft.fftfreq(n1)
    f2 = np.fft.fftfreq(n2)
    g = np.exp(-2.0 * (math.pi * sigma) ** 2 * (f1[:, None] ** 2 + f2[None, :] ** 2))
    return np.real(np.fft.ifft2(np.fft.fft2(a) * g))


def _rescale(a: np.ndarray, lo: float, hi: float) -> np.ndarray:
    amin, amax = a.min(), a.max()
    if amax - amin <= 0:
        return np.full_like(a, 0.5 * (lo + hi))
    return lo + (a - amin) * ((hi - lo) / (amax - amin))


def make_object(rng: np.random.Generator, n1: int, n2: int, *, amp=(0.6, 1.0),
                phase=(0.0, math.pi / 2), sigma=2.0) -> np.ndarray:
    a = _rescale(_smooth_periodic(rng.uniform(amp[0], amp[1], (n1, n2)), sigma), *amp)
    p = _rescale(_smooth_periodic(rng.uniform(phase[0], phase[1], (n1, n2)), sigma), *phase)
    return a * np.exp(1j * p)


def make_probe(rng: np.random.Generator, n_p: int, sigma: float) -> np.ndarray:
    c = (n_p - 1) / 2.0
    r = np.arange(n_p) - c
    r2 = r[:, None] ** 2 + r[None, :] ** 2
    amp = np.exp(-r2 / (2.0 * sigma * sigma))
    a = rng.uniform(0.0, 2.0 * math.pi)
    return amp * np.exp(1j * a * r2 / (n_p / 2.0) ** 2)


def make_offsets(rng: np.random.Generator, n_obj: int, n_p: int, n_scan: int,
                 step: int, jitter: int, n_obj2: int | None = None) -> np.ndarray:
    n_obj2 = n_obj if n_obj2 is None else n_obj2
    out = np.empty((n_scan * n_scan, 2), dtype=np.int32)
    m1 = (n_obj - (n_scan - 1) * step - n_p) // 2
    m2 = (n_obj2 - (n_scan - 1) * step - n_p) // 2
    k = 0
    for i in range(n_scan):
        for j in range(n_scan):
            dr, dc = rng.integers(-jitter, jitter + 1, size=2) if jitter > 0 else (0, 0)
            out[k, 0] = min(max(m1 + i * step + int(dr), 0), n_obj - n_p)
            out[k, 1] = min(max(m2 + j * step + int(dc), 0), n_obj2 - n_p)
            k += 1
    return out


def simulate(rng: np.random.Generator | None, x: np.ndarray, probe: np.ndarray,
             offsets: np.ndarray, peak: float | None, chunk: int = 256) -> np.ndarray:
    """Forward model of Section II plus the Section IV photon scaling."""
    n_p = probe.shape[0]
    J = offsets.shape[0]
    y = np.empty((J, n_p, n_p), dtype=np.float64)
    for s in range(0, J, chunk):
        e = min(J, s + chunk)
        fr = np.stack([probe * x[o[0]:o[0] + n_p, o[1]:o[1] + n_p] for o in offsets[s:e]])
        inten = np.abs(np.fft.fft2(fr, norm="ortho")) ** 2
        if peak is None:
            y[s:e] = np.sqrt(inten)
        else:
            m = inten.reshape(e - s, -1).max(axis=1)[:, None, None]
            m = np.where(m > 0, m, 1.0)
            counts = rng.poisson(inten * (peak / m))
            y[s:e] = np.sqrt(counts) * np.sqrt(m / peak)
    return y


def make_workload(config: str | dict = "small", seed: int = 1, *, noiseless=False,
                  peak: float | None = -1.0, n_scan: int | None = None) -> Workload:
    """Draw one workload.  `config` is a key of CONFIGS or an explicit dict."""
    c = dict(CONFIGS[config]) if isinstance(config, str) else dict(config)
    name = config if isinstance(config, str) else c.get("name", "custom")
    if n_scan is not None:
        c["n_scan"] = n_scan
    rng = np.random.Generator(np.random.PCG64(seed))
    x = make_object(rng, c["n_obj"], c.get("n_obj2", c["n_obj"]))
    probe = make_probe(rng, c["n_p"], c["probe_sigma"])
    offs = make_offsets(rng, c["n_obj"], c["n_p"], c["n_scan"], c["step"], c["jitter"],
                        c.get("n_obj2"))
    pk = None if noiseless else (c["peak"] if peak == -1.0 else peak)
    y = simulate(rng, x, probe, offs, pk)
    return Workload(name=name, x=x, probe=probe, offsets=offs, y=y, peak=pk, seed=seed)


def quantize_amplitudes_f16(y: np.ndarray):
    """Per-pattern FP16 storage: s_j = max(y_j), stored y_j / s_j in [0, 1].

    Returns (codes float16 (J,Np,Np), scales float32 (J,)).  The dequantized
    values codes * scales (exact in float64) are what the FP16 path solves.
    """
    J = y.shape[0]
    s = y.reshape(J, -1).max(axis=1).astype(np.float32)
    s = np.where(s > 0, s, np.float32(1.0)).astype(np.float32)
    codes = (y / s.astype(np.float64)[:, None, None]).astype(np.float16)
    return codes, s


def dequantize_f16(codes: np.ndarray, scales: np.ndarray) -> np.ndarray:
    return codes.astype(np.float64) * scales.astype(np.float64)[:, None, None]
