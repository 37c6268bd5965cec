"""Algorithm 1 of the FP64 oracle with the agent step taken over the whole
patch stack at once, on every host core.

TEST INFRASTRUCTURE ONLY: the benchmark's second CPU baseline (the literal
single-thread oracle is the first) and the tests that check it.  Nothing in
the product path imports it.

The arithmetic is that of oracle.pmace_oracle.pmace, in complex128, in the
paper's order (Algorithm 1: w <- F(v); z <- G(2w - v); v <- v + 2 rho (z -
w); x_hat = Lambda^-1 sum_j P_j^t |D|^kappa v_j).  Only the evaluation of
the agents differs: the closed form of Section III-A (equation
F-interpolate) is applied to all patches of an iteration together, with the
2-D orthonormal DFTs of the stack taken by one scipy.fft call that uses
`workers` threads.  The consensus G and the readout are the oracle's own
functions.  The residual sums of the literal oracle are not formed.
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft as sfft

from . import pmace_oracle as orc


def agents_batched(v: np.ndarray, y: np.ndarray, probe: np.ndarray, alpha: float,
                   workers: int) -> np.ndarray:
    """F_j applied to every patch of the stack v (Section III-A, equation
    F-interpolate), the phase factor 0 where F D v_j = 0 and the input
    returned where |d| <= TINY_PROBE max|d|."""
    a = sfft.fft2(probe[None] * v, norm="ortho", workers=workers)
    mag = np.abs(a)
    phase = np.zeros_like(a)
    np.divide(a, mag, out=phase, where=mag > 0)
    back = sfft.ifft2(y * phase, norm="ortho", workers=workers)
    ok = np.abs(probe) > orc.TINY_PROBE * np.abs(probe).max()
    out = v.astype(np.complex128).copy()
    out[:, ok] = (alpha * v[:, ok] + back[:, ok] / probe[ok]) / (1.0 + alpha)
    return out


def pmace(y: np.ndarray, probe: np.ndarray, offsets: np.ndarray, shape, *, alpha: float,
          rho: float = 0.5, kappa: float = 1.25, n_iter: int = 1, x0: np.ndarray | None = None,
          v0: np.ndarray | None = None, workers: int | None = None) -> dict:
    """Algorithm 1 from an image x0 (default: the energy-matched constant) or
    a patch stack v0; returns the final stacks v, w, z, the consensus image
    of the last step and x_hat."""
    workers = workers or os.cpu_count() or 1
    n_p = probe.shape[0]
    lam_inv = orc.inverse_weights(orc.weight_image(probe, offsets, shape, kappa))
    if v0 is None:
        v = orc.init_stack(orc.default_init(y, probe, shape) if x0 is None else x0, offsets, n_p)
    else:
        v = v0.astype(np.complex128).copy()
    w = z = v
    xbar = np.zeros(shape, dtype=np.complex128)
    for _ in range(n_iter):
        w = agents_batched(v, y, probe, alpha, workers)                         # w <- F(v)
        xbar = orc.consensus_image(2.0 * w - v, probe, offsets, lam_inv, kappa)
        z = orc.redistribute(xbar, offsets, n_p)                                # z <- G(2w - v)
        v = v + 2.0 * rho * (z - w)                                             # v <- v + 2 rho (z - w)
    return dict(v=v, w=w, z=z, xbar=xbar, x_hat=orc.readout(v, probe, offsets, lam_inv, kappa))
