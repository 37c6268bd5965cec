"""Plant plausible mistakes in a private copy of the oracle (on the CPU) and
check that at least one pin catches each.  This is how the pins are shown to
constrain every step of the oracle, not just to agree with it."""
import importlib.util
import os

import numpy as np
import pytest

from tests import oracle_pins

ORACLE_FILE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                           "oracle", "pmace_oracle.py")


def _fresh_copy(tag):
    spec = importlib.util.spec_from_file_location(f"_mutant_{tag}", ORACLE_FILE)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _m_probe_not_inverted(o):
    orig = o.agent

    def agent(xj, yj, probe, alpha):
        a = o.fft2o(probe * xj)
        mag = np.abs(a)
        ph = np.where(mag > 0, a / np.where(mag > 0, mag, 1), 0)
        return (alpha * xj + o.ifft2o(yj * ph) * np.conj(probe)) / (1 + alpha)
    o.agent = agent
    del orig


def _m_alpha_swapped(o):
    def agent(xj, yj, probe, alpha):
        a = o.fft2o(probe * xj)
        mag = np.abs(a)
        ph = np.where(mag > 0, a / np.where(mag > 0, mag, 1), 0)
        return (xj + alpha * o.ifft2o(yj * ph) / probe) / (1 + alpha)
    o.agent = agent


def _m_conj_phase(o):
    def agent(xj, yj, probe, alpha):
        a = o.fft2o(probe * xj)
        mag = np.abs(a)
        ph = np.where(mag > 0, np.conj(a) / np.where(mag > 0, mag, 1), 0)
        return (alpha * xj + o.ifft2o(yj * ph) / probe) / (1 + alpha)
    o.agent = agent


def _m_unnormalised_fft(o):
    o.fft2o = lambda a: np.fft.fft2(a)
    o.ifft2o = lambda a: np.fft.ifft2(a)


def _m_transposed_fft(o):
    o.fft2o = lambda a: np.swapaxes(np.fft.fft2(a, norm="ortho"), -1, -2)


def _m_no_kappa_in_numerator(o):
    def consensus_image(stack, probe, offsets, lam_inv, kappa):
        img = np.zeros(lam_inv.shape, dtype=np.complex128)
        for i in range(stack.shape[0]):
            o.backproject_add(img, stack[i], offsets[i])
        return img * lam_inv
    o.consensus_image = consensus_image


def _m_half_kappa_in_lambda(o):
    orig = o.weight_image
    o.weight_image = lambda probe, offsets, shape, kappa: orig(probe, offsets, shape, kappa / 2)


def _m_transposed_offsets(o):
    orig_e, orig_b = o.extract, o.backproject_add
    o.extract = lambda x, off, n_p: orig_e(x, (off[1], off[0]), n_p)
    o.backproject_add = lambda img, patch, off: orig_b(img, patch, (off[1], off[0]))


def _m_transposed_extract_only(o):
    orig_e = o.extract
    o.extract = lambda x, off, n_p: orig_e(x, (off[1], off[0]), n_p)


def _m_mann_sign(o):
    src = open(ORACLE_FILE).read().replace("v = v + 2.0 * rho * (z - w)", "v = v - 2.0 * rho * (z - w)")
    exec(compile(src, ORACLE_FILE, "exec"), o.__dict__)


def _m_consensus_of_w(o):
    src = open(ORACLE_FILE).read().replace("consensus_image(2.0 * w - v,", "consensus_image(w,")
    exec(compile(src, ORACLE_FILE, "exec"), o.__dict__)


def _m_readout_of_w(o):
    src = open(ORACLE_FILE).read().replace("x_hat = readout(v,", "x_hat = readout(w,")
    exec(compile(src, ORACLE_FILE, "exec"), o.__dict__)


def _m_nrmse_theta_sign(o):
    def nrmse(x_hat, x, mask=None):
        if mask is not None:
            x_hat, x = x_hat[mask], x[mask]
        th = -np.angle(np.vdot(x, x_hat))
        return float(np.linalg.norm(x_hat - np.exp(1j * th) * x) / np.linalg.norm(x))
    o.nrmse = nrmse


def _m_init_energy(o):
    def default_init(y, probe, shape):
        c = np.sqrt(np.sum(y ** 2) / np.sum(np.abs(probe) ** 2))
        return np.full(shape, c, dtype=np.complex128)
    o.default_init = default_init


def _m_lambda_sqrt(o):
    def inverse_weights(lam):
        return np.where(lam > 0, 1.0 / np.sqrt(np.where(lam > 0, lam, 1)), 0.0)
    o.inverse_weights = inverse_weights


def _replace_in_source(o, old, new):
    src = open(ORACLE_FILE).read()
    assert old in src, old
    exec(compile(src.replace(old, new), ORACLE_FILE, "exec"), o.__dict__)


def _m_absent_probe_returns_zero(o):
    _replace_in_source(o, "out = xj.astype(np.complex128).copy()", "out = np.zeros(xj.shape, dtype=np.complex128)")


def _m_absent_probe_blended(o):
    _replace_in_source(o, "out = xj.astype(np.complex128).copy()",
                       "out = (alpha * xj / (1.0 + alpha)).astype(np.complex128)")


def _m_absent_probe_absolute_threshold(o):
    _replace_in_source(o, "ok = np.abs(probe) > TINY_PROBE * amax", "ok = np.abs(probe) > TINY_PROBE")


MUTATIONS = [_m_probe_not_inverted, _m_alpha_swapped, _m_conj_phase, _m_unnormalised_fft,
             _m_transposed_fft, _m_no_kappa_in_numerator, _m_half_kappa_in_lambda,
             _m_transposed_offsets, _m_transposed_extract_only, _m_mann_sign,
             _m_consensus_of_w, _m_readout_of_w, _m_nrmse_theta_sign, _m_init_energy,
             _m_lambda_sqrt, _m_absent_probe_returns_zero, _m_absent_probe_blended,
             _m_absent_probe_absolute_threshold]


@pytest.mark.parametrize("mutate", MUTATIONS, ids=lambda f: f.__name__[3:])
def test_pins_catch_mutation(mutate):
    o = _fresh_copy(mutate.__name__)
    mutate(o)
    caught = []
    for pin in oracle_pins.ALL_PINS:
        try:
            with np.errstate(all="ignore"):
                pin(o)
        except Exception:
            caught.append(pin.__name__)
    assert caught, f"no pin detects mutation {mutate.__name__}"
