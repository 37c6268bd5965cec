"""FP64 CPU oracle for PMACE (Zhai, Buzzard, Wohlberg, Bouman, arXiv 2111.14240).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or runs
this file: only the tests, the smoke check and the CPU-baseline leg of the
benchmark do.  It shares no code with the CUDA path; both are fed the same
seeded inputs by a separate generator module.

It is a plain, slow, literal restatement of the paper in complex128:

* the probe-weighted proximal agent F_j, closed form of Section III-A
  (equation "F-interpolate"), with the phase factor set to 0 where the
  Fourier transform vanishes (Section III-A, definition of u = r * w/|w|);
* the probe-weighted consensus G and the weight image Lambda (Section III-A,
  equation "xjbar");
* Algorithm 1 (Mann iteration for the PMACE solution), step by step in the
  paper's order: w <- F(v); z <- G(2w - v); v <- v + 2 rho (z - w); and the
  final weighted average x_hat = Lambda^-1 sum_j P_j^t |D|^kappa v_j;
* the NRMSE with the global phase chosen to minimise the error (Section IV).

Readings of points the paper leaves open (all mirrored in the CUDA path):

* the Fourier transform is the 2-D orthonormal DFT with the DC term at index
  0 (Section II names F the orthonormal transform);
* pixels no window covers have Lambda = 0; there Lambda^-1 := 0, so they
  read out as 0 and are excluded from the NRMSE mask;
* where |d| <= 1e-30 * max|d| the inverse D^-1 does not exist; the agent
  returns its input at such pixels (the alpha -> infinity limit there);
* residuals reported after an iteration t (the paper only says "while not
  converged"): r_fp = ||z_{t-1} - w_t|| / ||w_t||, the disagreement between
  the previous consensus and the new agent outputs (z_0 := v_0, the shared
  initialisation of Algorithm 1), which is zero exactly at the Algorithm 1
  fixed point; and r_data = sum_j ||y_j - |F D v_{t-1}| ||^2 / sum_j ||y_j||^2,
  the data term of equation "eq1" (up to 1/(2 sigma_n^2)) at the agents'
  inputs.

Parity pins: every function here is checked in tests/test_oracle_pins.py
against something other than itself (naive DFT, Parseval, exact magnitude,
idempotence of G, alpha limits, the noiseless fixed point, the G = I
reduction, phase equivariance, permutation invariance, brute-force NRMSE
phase).  The multi-iteration trajectory at a given alpha has no independent
pin beyond those invariants.
"""
from __future__ import annotations

import numpy as np

TINY_PROBE = 1e-30  # relative threshold below which D^-1 is treated as absent


# ---------------------------------------------------------------- transforms
def fft2o(a: np.ndarray) -> np.ndarray:
    """2-D orthonormal DFT over the last two axes (Section II)."""
    return np.fft.fft2(a, norm="ortho")


def ifft2o(a: np.ndarray) -> np.ndarray:
    """Adjoint (= inverse) of fft2o."""
    return np.fft.ifft2(a, norm="ortho")


# ---------------------------------------------------------------- projections
def extract(x: np.ndarray, off, n_p: int) -> np.ndarray:
    """P_j: the n_p x n_p window of x whose top-left corner is `off` (Section II)."""
    r, c = int(off[0]), int(off[1])
    return x[r:r + n_p, c:c + n_p].copy()


def backproject_add(img: np.ndarray, patch: np.ndarray, off) -> None:
    """img += P_j^t patch (the transpose of extract)."""
    n_p = patch.shape[0]
    r, c = int(off[0]), int(off[1])
    img[r:r + n_p, c:c + n_p] += patch


def weight_image(probe: np.ndarray, offsets: np.ndarray, shape, kappa: float) -> np.ndarray:
    """Lambda = sum_j P_j^t |D|^kappa (Section III-A, below equation xjbar)."""
    lam = np.zeros(shape, dtype=np.float64)
    wk = np.abs(probe) ** kappa
    for off in offsets:
        backproject_add(lam, wk, off)
    return lam


def inverse_weights(lam: np.ndarray) -> np.ndarray:
    """Lambda^-1 with the reading Lambda^-1 := 0 where Lambda = 0."""
    out = np.zeros_like(lam)
    nz = lam > 0
    out[nz] = 1.0 / lam[nz]
    return out


# ---------------------------------------------------------------- agent F_j
def agent(xj: np.ndarray, yj: np.ndarray, probe: np.ndarray, alpha: float) -> np.ndarray:
    """Probe-weighted proximal map F_j (Section III-A, equation F-interpolate).

    F_j(x_j) = (alpha x_j + D^-1 F^* (y_j * F D x_j / |F D x_j|)) / (1 + alpha),
    with the phase factor F D x_j / |F D x_j| taken as 0 where F D x_j = 0.
    """
    a = fft2o(probe * xj)
    mag = np.abs(a)
    phase = np.zeros_like(a)
    nz = mag > 0
    phase[nz] = a[nz] / mag[nz]
    back = ifft2o(yj * phase)
    amax = np.abs(probe).max()
    ok = np.abs(probe) > TINY_PROBE * amax
    out = xj.astype(np.complex128).copy()
    out[ok] = (alpha * xj[ok] + back[ok] / probe[ok]) / (1.0 + alpha)
    return out


def agents(v: np.ndarray, y: np.ndarray, probe: np.ndarray, alpha: float) -> np.ndarray:
    """Stacked F (Section III-A): F_j applied to every patch independently."""
    return np.stack([agent(v[j], y[j], probe, alpha) for j in range(v.shape[0])])


# ---------------------------------------------------------------- consensus G
def consensus_image(stack: np.ndarray, probe: np.ndarray, offsets: np.ndarray,
                    lam_inv: np.ndarray, kappa: float) -> np.ndarray:
    """Lambda^-1 sum_i P_i^t |D|^kappa x_i (the full image inside equation xjbar)."""
    img = np.zeros(lam_inv.shape, dtype=np.complex128)
    wk = np.abs(probe) ** kappa
    for i in range(stack.shape[0]):
        backproject_add(img, wk * stack[i], offsets[i])
    return img * lam_inv


def redistribute(img: np.ndarray, offsets: np.ndarray, n_p: int) -> np.ndarray:
    """[P_j img]_j: the stack of windows of an image."""
    return np.stack([extract(img, o, n_p) for o in offsets])


def consensus(stack: np.ndarray, probe: np.ndarray, offsets: np.ndarray,
              lam_inv: np.ndarray, kappa: float) -> np.ndarray:
    """G (Section III-A, equation xjbar): xbar_j = P_j Lambda^-1 sum_i P_i^t |D|^kappa x_i."""
    img = consensus_image(stack, probe, offsets, lam_inv, kappa)
    return redistribute(img, offsets, probe.shape[0])


# ---------------------------------------------------------------- Algorithm 1
def init_stack(x0: np.ndarray, offsets: np.ndarray, n_p: int) -> np.ndarray:
    """Algorithm 1 initialisation: w = v = [P_j x^(0)]_j."""
    return redistribute(x0.astype(np.complex128), offsets, n_p)


def default_init(y: np.ndarray, probe: np.ndarray, shape) -> np.ndarray:
    """Energy-matched constant start: c = sqrt(sum_j ||y_j||^2 / (J ||d||^2)).

    By Parseval (F orthonormal, Section II) a constant patch c gives
    ||F D c|| = c ||d||, so this c matches the measured energy on average.
    """
    J = y.shape[0]
    c = np.sqrt(np.sum(y.astype(np.float64) ** 2) / (J * np.sum(np.abs(probe) ** 2)))
    return np.full(shape, c, dtype=np.complex128)


def readout(v: np.ndarray, probe: np.ndarray, offsets: np.ndarray,
            lam_inv: np.ndarray, kappa: float) -> np.ndarray:
    """Algorithm 1 output: x_hat = Lambda^-1 sum_j P_j^t |D|^kappa v_j."""
    return consensus_image(v, probe, offsets, lam_inv, kappa)


def pmace(y: np.ndarray, probe: np.ndarray, offsets: np.ndarray, shape, *,
          alpha: float, rho: float = 0.5, kappa: float = 1.25, n_iter: int = 1,
          x0: np.ndarray | None = None, v0: np.ndarray | None = None,
          z_prev: np.ndarray | None = None, record: bool = False) -> dict:
    """Algorithm 1 (Mann iteration for the PMACE solution), literally.

    Either start from an image x0 (default: energy-matched constant) or from a
    given patch stack v0.  Returns the final stacks v, w, z, the consensus
    image of the last step, x_hat, and the residuals of the last iteration.
    """
    n_p = probe.shape[0]
    lam_inv = inverse_weights(weight_image(probe, offsets, shape, kappa))
    if v0 is None:
        if x0 is None:
            x0 = default_init(y, probe, shape)
        v = init_stack(x0, offsets, n_p)
    else:
        v = v0.astype(np.complex128).copy()
    w = v.copy()
    z = v.copy() if z_prev is None else z_prev.astype(np.complex128).copy()
    xbar = np.zeros(shape, dtype=np.complex128)
    history = []
    r_fp = r_data = None
    for _ in range(n_iter):
        z_before = z
        # residual of the data term at the agents' inputs (equation eq1)
        fr = np.abs(fft2o(probe[None] * v))
        r_data = float(np.sum((y - fr) ** 2) / np.sum(y.astype(np.float64) ** 2))
        w = agents(v, y, probe, alpha)                       # w <- F(v)
        xbar = consensus_image(2.0 * w - v, probe, offsets, lam_inv, kappa)
        z = redistribute(xbar, offsets, n_p)                 # z <- G(2w - v)
        v = v + 2.0 * rho * (z - w)                          # v <- v + 2 rho (z - w)
        r_fp = float(np.sqrt(np.sum(np.abs(z_before - w) ** 2) / np.sum(np.abs(w) ** 2)))
        if record:
            history.append(dict(r_fp=r_fp, r_data=r_data))
    x_hat = readout(v, probe, offsets, lam_inv, kappa)
    return dict(v=v, w=w, z=z, xbar=xbar, x_hat=x_hat, lam_inv=lam_inv,
                r_fp=r_fp, r_data=r_data, history=history)


# ---------------------------------------------------------------- evaluation
def nrmse(x_hat: np.ndarray, x: np.ndarray, mask: np.ndarray | None = None) -> float:
    """Section IV: e = ||x_hat - e^{i theta} x|| / ||x||, theta minimising the numerator.

    ||x_hat - e^{i t} x||^2 = ||x_hat||^2 + ||x||^2 - 2 Re(e^{-i t} <x, x_hat>) with
    <x, x_hat> = sum conj(x) x_hat, minimised at t = arg <x, x_hat>.
    """
    if mask is not None:
        x_hat = x_hat[mask]
        x = x[mask]
    theta = np.angle(np.vdot(x, x_hat))
    return float(np.linalg.norm(x_hat - np.exp(1j * theta) * x) / np.linalg.norm(x))
