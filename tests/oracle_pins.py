"""Pins for the FP64 oracle: checks against things other than the oracle itself.

Each pin takes the oracle module as its argument so that the same checks can
be run against deliberately broken copies of it (tests/test_oracle_mutations.py)
to show that a plausible mistake anywhere in the oracle fails at least one pin.

References are to the paper's sections and equation labels
(Zhai et al., arXiv 2111.14240).
"""
from __future__ import annotations

import cmath
import math

import numpy as np

from paper_2111_14240_gb300 import datagen


def _rng(seed=0):
    return np.random.Generator(np.random.PCG64(seed))


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _tiny_scan(seed=3, n_obj=24, n_p=8, n_scan=4, step=5, jitter=1):
    rng = _rng(seed)
    x = datagen.make_object(rng, n_obj, n_obj)
    d = datagen.make_probe(rng, n_p, n_p / 4)
    offs = datagen.make_offsets(rng, n_obj, n_p, n_scan, step, jitter)
    return x, d, offs


# ------------------------------------------------------------------ T1, T2
def naive_dft2(a):
    """Orthonormal 2-D DFT written out as the quadruple sum (Section II: F orthonormal)."""
    n1, n2 = a.shape
    out = np.zeros((n1, n2), dtype=complex)
    for k1 in range(n1):
        for k2 in range(n2):
            s = 0j
            for m1 in range(n1):
                for m2 in range(n2):
                    s += a[m1, m2] * cmath.exp(-2j * math.pi * (k1 * m1 / n1 + k2 * m2 / n2))
            out[k1, k2] = s / math.sqrt(n1 * n2)
    return out


def pin_fft_naive(o):
    """T1: the oracle's transform equals the naive orthonormal DFT (4x4, 8x8, 4x8, 16x16)."""
    rng = _rng(1)
    for shape in [(4, 4), (8, 8), (4, 8), (16, 16)]:
        a = _crandn(rng, *shape)
        ref = naive_dft2(a)
        assert np.max(np.abs(o.fft2o(a) - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))
        # and its inverse undoes it
        assert np.max(np.abs(o.ifft2o(ref) - a)) < 1e-12 * np.max(np.abs(a))


def pin_parseval(o):
    """T2: ||F a|| = ||a|| for the orthonormal transform."""
    rng = _rng(2)
    a = _crandn(rng, 32, 32)
    assert abs(np.linalg.norm(o.fft2o(a)) - np.linalg.norm(a)) < 1e-12 * np.linalg.norm(a)


# ------------------------------------------------------------------ agent
def pin_agent_scalar(o):
    """1x1 patches: F is the identity, so equation F-interpolate reduces to
    (alpha x + (1/d) y (d x)/|d x|) / (1 + alpha), checked in scalars."""
    rng = _rng(4)
    for _ in range(20):
        x = complex(*rng.standard_normal(2))
        d = complex(*rng.standard_normal(2))
        y = abs(rng.standard_normal()) + 0.1
        alpha = float(rng.uniform(0.0, 3.0))
        dx = d * x
        expect = (alpha * x + (1.0 / d) * y * dx / abs(dx)) / (1.0 + alpha)
        got = o.agent(np.array([[x]]), np.array([[y]]), np.array([[d]]), alpha)[0, 0]
        assert abs(got - expect) < 1e-12 * max(1.0, abs(expect))


def pin_agent_magnitude(o):
    """T3 / T5 (alpha = 0): the returned patch fits the data exactly,
    |F D F_j(x)| = y wherever F D x != 0 (Section III-A)."""
    rng = _rng(5)
    n = 16
    d = datagen.make_probe(rng, n, 4.0)
    x = _crandn(rng, n, n)
    y = np.abs(rng.standard_normal((n, n))) + 0.05
    w = o.agent(x, y, d, 0.0)
    assert np.max(np.abs(np.abs(np.fft.fft2(d * w, norm="ortho")) - y)) < 1e-10
    # and the phase of F D w is that of F D x
    a0 = np.fft.fft2(d * x, norm="ortho")
    a1 = np.fft.fft2(d * w, norm="ortho")
    assert np.max(np.abs(a1 / np.abs(a1) - a0 / np.abs(a0))) < 1e-10


def pin_agent_zero_phase(o):
    """T3: where F D x = 0 the phase factor is 0 (Section III-A).  A zero patch
    has an exactly zero transform, so the agent must return exactly 0 (not
    NaN) for any y and alpha; on a 1x1 window a zero value maps to 0 too."""
    rng = _rng(6)
    n = 8
    d = datagen.make_probe(rng, n, 2.0)
    y = np.abs(rng.standard_normal((n, n))) + 1.0
    for alpha in (0.0, 0.5):
        w = o.agent(np.zeros((n, n), dtype=complex), y, d, alpha)
        assert np.all(w == 0)
    w1 = o.agent(np.array([[0j]]), np.array([[2.0]]), np.array([[0.5 + 0.5j]]), 0.0)
    assert w1[0, 0] == 0


def pin_agent_alpha_limits(o):
    """T5 (Section III-A): alpha -> infinity returns the input; the alpha
    blend is linear: F_alpha = (alpha x + F_0(x)) / (1 + alpha)."""
    rng = _rng(7)
    n = 16
    d = datagen.make_probe(rng, n, 4.0)
    x = _crandn(rng, n, n)
    y = np.abs(rng.standard_normal((n, n)))
    assert np.max(np.abs(o.agent(x, y, d, 1e12) - x)) < 1e-9
    f0 = o.agent(x, y, d, 0.0)
    for alpha in (0.3, 2.0):
        assert np.max(np.abs(o.agent(x, y, d, alpha) - (alpha * x + f0) / (1 + alpha))) < 1e-11


def pin_agent_variational(o):
    """The agent solves the proximal problem of equation Fjv:
    F_j(x) = argmin_v 0.5||y - |F D v| ||^2 + 0.5 alpha ||F D v - F D x||^2
    (both terms scaled by sigma_n^2, alpha = sigma_n^2 / sigma^2).  Checked by
    (a) the pointwise minimiser r* = (alpha|w| + y)/(alpha + 1) of the
    magnitude problem found by a dense scan, and (b) random perturbations of
    the returned v never lowering the objective."""
    rng = _rng(8)
    n = 8
    d = datagen.make_probe(rng, n, 2.0)
    x = _crandn(rng, n, n)
    y = np.abs(rng.standard_normal((n, n))) + 0.1
    alpha = 0.7

    def obj(v):
        a = np.fft.fft2(d * v, norm="ortho")
        b = np.fft.fft2(d * x, norm="ortho")
        return 0.5 * np.sum((y - np.abs(a)) ** 2) + 0.5 * alpha * np.sum(np.abs(a - b) ** 2)

    v = o.agent(x, y, d, alpha)
    # (a) magnitude of F D v is the scalar minimiser, computed by a scan
    wabs = np.abs(np.fft.fft2(d * x, norm="ortho"))
    got = np.abs(np.fft.fft2(d * v, norm="ortho"))
    for (i, j) in [(0, 0), (1, 3), (5, 2), (7, 7)]:
        rs = np.linspace(0, 3 * max(y[i, j], wabs[i, j]) + 1, 200001)
        best = rs[np.argmin(0.5 * (rs - y[i, j]) ** 2 + 0.5 * alpha * (rs - wabs[i, j]) ** 2)]
        assert abs(got[i, j] - best) < 1e-4 * (1 + best)
    # (b) local optimality
    f0 = obj(v)
    for _ in range(50):
        dv = _crandn(rng, n, n) * 1e-3
        assert obj(v + dv) >= f0 - 1e-12


def naive_idft2(a):
    """Inverse of naive_dft2: the adjoint of the orthonormal DFT, conj(F conj(a))."""
    return np.conj(naive_dft2(np.conj(a)))


def pin_agent_absent_probe(o):
    """Pixels where the probe vanishes.  D^-1 in equation F-interpolate is
    undefined there; the reading taken is that where |d| <= 1e-30 max|d| the
    agent returns its input at that pixel (the alpha -> infinity limit of
    that pixel), for every alpha.  Checked against the closed form written
    with the naive DFT:
    (a) 1x1 windows with d = 0 return x exactly;
    (b) an 8x8 window whose probe has exact zeros, a pixel at 0.5e-30 of the
        peak (absent) and one at 2e-30 (present): absent pixels return x bit
        for bit, every other pixel is (alpha x + (F^* y F D x / |F D x|) / d)
        / (1 + alpha);
    (c) the threshold is relative to the peak: the same probe scaled by
        1e-40 obeys (b) with the scaled d."""
    rng = _rng(9)
    for alpha in (0.0, 0.5, 3.0):
        x = complex(*rng.standard_normal(2))
        got = o.agent(np.array([[x]]), np.array([[1.7]]), np.array([[0j]]), alpha)[0, 0]
        assert got == x
    n = 8
    d = datagen.make_probe(rng, n, 2.0)
    amax = np.abs(d).max()
    absent = [(0, 0), (0, 5), (7, 7), (3, 6)]
    for p in absent[:3]:
        d[p] = 0.0
    d[3, 6] = 0.5e-30 * amax * np.exp(0.3j)
    d[6, 1] = 2e-30 * amax * np.exp(-1.1j)
    assert np.abs(d).max() == amax
    for scale in (1.0, 1e-40):
        ds = d * scale
        x = _crandn(rng, n, n)
        y = np.abs(rng.standard_normal((n, n))) + 0.2
        a = naive_dft2(ds * x)
        back = naive_idft2(y * a / np.abs(a))
        for alpha in (0.0, 0.7, 4.0):
            got = o.agent(x, y, ds, alpha)
            for i in range(n):
                for k in range(n):
                    if (i, k) in absent:
                        assert got[i, k] == x[i, k], (scale, alpha, i, k)
                    else:
                        expect = (alpha * x[i, k] + back[i, k] / ds[i, k]) / (1.0 + alpha)
                        assert abs(got[i, k] - expect) <= 1e-9 * abs(expect), (scale, alpha, i, k)


# ------------------------------------------------------------------ consensus
def pin_weight_image_bruteforce(o):
    """Lambda(p) = sum over windows containing p of |d(p - o_j)|^kappa, written
    pixel by pixel (Section III-A, below equation xjbar)."""
    x, d, offs = _tiny_scan()
    n_p = d.shape[0]
    kappa = 1.25
    lam = o.weight_image(d, offs, x.shape, kappa)
    ref = np.zeros(x.shape)
    for p1 in range(x.shape[0]):
        for p2 in range(x.shape[1]):
            for (r, c) in offs:
                if r <= p1 < r + n_p and c <= p2 < c + n_p:
                    ref[p1, p2] += abs(d[p1 - r, p2 - c]) ** kappa
    assert np.max(np.abs(lam - ref)) < 1e-12


def pin_consensus_bruteforce(o):
    """G written per pixel as a weighted average of every patch value covering
    it, weights |d|^kappa (equation xjbar), then redistributed."""
    x, d, offs = _tiny_scan(seed=9)
    n_p = d.shape[0]
    kappa = 1.25
    rng = _rng(10)
    stack = _crandn(rng, len(offs), n_p, n_p)
    lam_inv = o.inverse_weights(o.weight_image(d, offs, x.shape, kappa))
    got = o.consensus(stack, d, offs, lam_inv, kappa)
    img = np.zeros(x.shape, dtype=complex)
    for p1 in range(x.shape[0]):
        for p2 in range(x.shape[1]):
            num, den = 0j, 0.0
            for j, (r, c) in enumerate(offs):
                if r <= p1 < r + n_p and c <= p2 < c + n_p:
                    wgt = abs(d[p1 - r, p2 - c]) ** kappa
                    num += wgt * stack[j, p1 - r, p2 - c]
                    den += wgt
            img[p1, p2] = num / den if den > 0 else 0
    ref = np.stack([img[r:r + n_p, c:c + n_p] for (r, c) in offs])
    assert np.max(np.abs(got - ref)) < 1e-12


def pin_consensus_idempotent(o):
    """T4: G(G(x)) = G(x), and G([P_j x]) = [P_j x] (consistent stacks are fixed)."""
    x, d, offs = _tiny_scan(seed=11)
    n_p = d.shape[0]
    kappa = 1.25
    rng = _rng(12)
    stack = _crandn(rng, len(offs), n_p, n_p)
    lam_inv = o.inverse_weights(o.weight_image(d, offs, x.shape, kappa))
    g1 = o.consensus(stack, d, offs, lam_inv, kappa)
    g2 = o.consensus(g1, d, offs, lam_inv, kappa)
    assert np.max(np.abs(g1 - g2)) < 1e-12
    px = np.stack([x[r:r + n_p, c:c + n_p] for (r, c) in offs])
    assert np.max(np.abs(o.consensus(px, d, offs, lam_inv, kappa) - px)) < 1e-12


# ------------------------------------------------------------------ Algorithm 1
def _noiseless(seed=13, n_obj=24, n_p=8, n_scan=4, step=5, jitter=1):
    x, d, offs = _tiny_scan(seed, n_obj, n_p, n_scan, step, jitter)
    y = datagen.simulate(None, x, d, offs, None)
    return x, d, offs, y


def pin_fixed_point(o):
    """T6: with noiseless data the ground truth is a fixed point of Algorithm 1
    (w = v, z = v, v unchanged) and the output is the ground truth on every
    covered pixel; the same holds for e^{i theta} x."""
    x, d, offs, y = _noiseless()
    n_p = d.shape[0]
    for th in (0.0, 1.1):
        xs = x * np.exp(1j * th)
        v0 = np.stack([xs[r:r + n_p, c:c + n_p] for (r, c) in offs])
        res = o.pmace(y, d, offs, x.shape, alpha=0.8, rho=0.5, n_iter=3, v0=v0)
        assert np.max(np.abs(res["v"] - v0)) < 1e-12
        assert np.max(np.abs(res["w"] - v0)) < 1e-12
        cov = o.weight_image(d, offs, x.shape, 1.25) > 0
        assert np.max(np.abs(res["x_hat"][cov] - xs[cov])) < 1e-12
        assert res["r_fp"] < 1e-12 and res["r_data"] < 1e-24


def pin_tiling_reduces_to_agent(o):
    """T7: non-overlapping windows make G the identity on stacks, and with
    rho = 1/2 Algorithm 1's update v <- v + (z - w) = 2w - v - w + v becomes
    v <- F(v).  Compared with the per-patch closed form written here."""
    rng = _rng(14)
    n_p, n = 8, 3
    d = datagen.make_probe(rng, n_p, 2.0)
    offs = np.array([(r * n_p, c * n_p) for r in range(n) for c in range(n)], dtype=np.int32)
    y = np.abs(rng.standard_normal((n * n, n_p, n_p))) + 0.1
    v0 = _crandn(rng, n * n, n_p, n_p)
    alpha = 0.6
    res = o.pmace(y, d, offs, (n * n_p, n * n_p), alpha=alpha, rho=0.5, n_iter=2, v0=v0)
    v = v0.copy()
    for _ in range(2):
        a = np.fft.fft2(d * v, norm="ortho")
        v = (alpha * v + np.fft.ifft2(y * a / np.abs(a), norm="ortho") / d) / (1 + alpha)
    assert np.max(np.abs(res["v"] - v)) < 1e-11


def pin_phase_equivariance(o):
    """T8: the measurements do not see a global phase, so the iteration
    commutes with it: iterate(e^{i t} v) = e^{i t} iterate(v)."""
    x, d, offs = _tiny_scan(seed=15)
    n_p = d.shape[0]
    rng = _rng(16)
    y = np.abs(rng.standard_normal((len(offs), n_p, n_p))) + 0.1
    v0 = _crandn(rng, len(offs), n_p, n_p)
    t = 0.77
    a = o.pmace(y, d, offs, x.shape, alpha=0.5, rho=0.4, n_iter=3, v0=v0)
    b = o.pmace(y, d, offs, x.shape, alpha=0.5, rho=0.4, n_iter=3, v0=v0 * np.exp(1j * t))
    assert np.max(np.abs(b["x_hat"] - np.exp(1j * t) * a["x_hat"])) < 1e-11


def pin_permutation_invariance(o):
    """T9: the agents are independent and G is a sum over patches, so
    permuting the patch order permutes the stacks and leaves x_hat unchanged."""
    x, d, offs = _tiny_scan(seed=17)
    n_p = d.shape[0]
    rng = _rng(18)
    y = np.abs(rng.standard_normal((len(offs), n_p, n_p))) + 0.1
    v0 = _crandn(rng, len(offs), n_p, n_p)
    perm = rng.permutation(len(offs))
    a = o.pmace(y, d, offs, x.shape, alpha=0.5, rho=0.5, n_iter=3, v0=v0)
    b = o.pmace(y[perm], d, offs[perm], x.shape, alpha=0.5, rho=0.5, n_iter=3, v0=v0[perm])
    assert np.max(np.abs(b["x_hat"] - a["x_hat"])) < 1e-11
    assert np.max(np.abs(b["v"] - a["v"][perm])) < 1e-11


def pin_mann_step_explicit(o):
    """One Algorithm 1 step written out with the brute-force G and the scalar
    agent on 1x1 windows (where F is the identity); checks the order
    w <- F(v), z <- G(2w - v), v <- v + 2 rho (z - w) and that the output
    averages the final v (not w or z)."""
    rng = _rng(19)
    # 1x1 windows on a 3x3 image, two windows per pixel for the first row
    offs = np.array([(0, 0), (0, 0), (0, 1), (0, 1), (1, 2), (2, 2)], dtype=np.int32)
    d = np.array([[0.8 - 0.3j]])
    y = np.abs(rng.standard_normal((6, 1, 1))) + 0.2
    v0 = _crandn(rng, 6, 1, 1)
    alpha, rho, kappa = 0.4, 0.3, 1.25
    res = o.pmace(y, d, offs, (3, 3), alpha=alpha, rho=rho, kappa=kappa, n_iter=1, v0=v0)
    dd = d[0, 0]
    v = v0[:, 0, 0]
    w = np.array([(alpha * v[j] + (1 / dd) * y[j, 0, 0] * (dd * v[j]) / abs(dd * v[j]))
                  / (1 + alpha) for j in range(6)])
    u = 2 * w - v
    z = np.empty(6, dtype=complex)
    for j, (r, c) in enumerate(offs):
        same = [i for i, (r2, c2) in enumerate(offs) if (r2, c2) == (r, c)]
        z[j] = np.mean(u[same])   # equal weights |d|^kappa on a shared 1x1 window
    vn = v + 2 * rho * (z - w)
    assert np.max(np.abs(res["v"][:, 0, 0] - vn)) < 1e-12
    assert np.max(np.abs(res["z"][:, 0, 0] - z)) < 1e-12
    # output: the (equal-weight) average of the final v over each window
    xh = np.zeros((3, 3), dtype=complex)
    for (r, c) in set(map(tuple, offs)):
        same = [i for i, (r2, c2) in enumerate(offs) if (r2, c2) == (r, c)]
        xh[r, c] = np.mean(vn[same])
    assert np.max(np.abs(res["x_hat"] - xh)) < 1e-12


def pin_readout(o):
    """Algorithm 1 output: for a consistent stack [P_j x], x_hat = x on covered
    pixels and 0 on uncovered ones (reading Lambda^-1 := 0)."""
    x, d, offs = _tiny_scan(seed=20, n_obj=30)   # leaves an uncovered border
    n_p = d.shape[0]
    lam = o.weight_image(d, offs, x.shape, 1.25)
    lam_inv = o.inverse_weights(lam)
    px = np.stack([x[r:r + n_p, c:c + n_p] for (r, c) in offs])
    xh = o.readout(px, d, offs, lam_inv, 1.25)
    cov = lam > 0
    assert (~cov).any()
    assert np.max(np.abs(xh[cov] - x[cov])) < 1e-12
    assert np.all(xh[~cov] == 0)


def pin_default_init(o):
    """Energy-matched start: with the constant c, sum_j ||F D P_j c||^2 =
    sum_j ||y_j||^2 (Parseval), computed here with numpy's FFT."""
    x, d, offs, y = _noiseless(seed=21)
    x0 = o.default_init(y, d, x.shape)
    n_p = d.shape[0]
    e = sum(np.sum(np.abs(np.fft.fft2(d * x0[r:r + n_p, c:c + n_p], norm="ortho")) ** 2)
            for (r, c) in offs)
    assert abs(e - np.sum(y ** 2)) < 1e-10 * np.sum(y ** 2)
    assert np.allclose(x0, x0.flat[0])


def pin_residual_definitions(o):
    """r_data is the data term of equation eq1 at the agents' inputs; written out."""
    x, d, offs = _tiny_scan(seed=22)
    n_p = d.shape[0]
    rng = _rng(23)
    y = np.abs(rng.standard_normal((len(offs), n_p, n_p))) + 0.1
    v0 = _crandn(rng, len(offs), n_p, n_p)
    res = o.pmace(y, d, offs, x.shape, alpha=0.5, rho=0.5, n_iter=1, v0=v0)
    num = sum(np.sum((y[j] - np.abs(np.fft.fft2(d * v0[j], norm="ortho"))) ** 2)
              for j in range(len(offs)))
    assert abs(res["r_data"] - num / np.sum(y ** 2)) < 1e-12
    w = res["w"]
    assert abs(res["r_fp"] - np.linalg.norm(v0 - w) / np.linalg.norm(w)) < 1e-12


# ------------------------------------------------------------------ NRMSE
def pin_nrmse_bruteforce(o):
    """T10: the closed-form theta matches a dense scan of theta in [0, 2 pi)."""
    rng = _rng(24)
    x = _crandn(rng, 12, 12)
    xh = x * np.exp(1j * 2.3) + 0.1 * _crandn(rng, 12, 12)
    got = o.nrmse(xh, x)
    ths = np.linspace(0, 2 * math.pi, 200001)
    ip = np.vdot(x, xh)
    errs = np.sqrt(np.maximum(np.sum(np.abs(xh) ** 2) + np.sum(np.abs(x) ** 2)
                              - 2 * np.real(np.exp(-1j * ths) * ip), 0)) / np.linalg.norm(x)
    assert abs(got - errs.min()) < 1e-6
    assert got < np.linalg.norm(xh - x) / np.linalg.norm(x)


def pin_convergence(o):
    """T11: on noiseless data with heavy overlap, from the constant start, the
    NRMSE falls monotonically and reaches the ground truth (< 1e-3 at 100 it)."""
    x, d, offs, y = _noiseless(seed=25, n_obj=32, n_p=16, n_scan=5, step=4, jitter=1)
    cov = o.weight_image(d, offs, x.shape, 1.25) > 0
    e = []
    v = None
    for _ in range(4):
        r = o.pmace(y, d, offs, x.shape, alpha=0.5, rho=0.5, n_iter=25, v0=v)
        v = r["v"]
        e.append(o.nrmse(r["x_hat"], x, cov))
    assert all(b < a for a, b in zip(e, e[1:])), e
    assert e[-1] < 1e-3, e


ALL_PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]
