"""Planted mistakes in the oracle's multi-determinant trial, each of which must fail at least one
of the pins in test_oracle_multidet.py (the control, no mutant, passes them all)."""
import numpy as np
import pytest

import test_oracle_multidet as P
from oracle import afqmc

ORIG = {n: getattr(afqmc, n) for n in ("det_shares", "green", "local_energy", "det_overlap")}

PINS = [
    ("overlap vs many-body vector", lambda: P.test_overlap_is_many_body_overlap(2, 1)),
    ("G as log-overlap derivative", lambda: P.test_green_function_is_log_overlap_derivative(2, 1)),
    ("rhobar as log-overlap derivative", P.test_force_bias_is_log_overlap_derivative),
    ("E_L vs dense H", lambda: P.test_local_energy_is_many_body_mixed_estimate(2, 1)),
    ("zero-variance trial", P.test_exact_ground_state_trial_has_zero_variance_local_energy),
]


def _shares(weight):
    def shares(sys, phi):
        logO = np.array([afqmc.det_overlap(sys, D, phi) for D in sys.dets])
        top = np.max(logO.real, axis=0)
        t = weight(sys.coeffs)[:, None] * np.exp(logO - top[None, :])
        total = np.sum(t, axis=0)
        return top + np.log(total), t / total[None, :]
    return shares


def _shares_unnormalised(sys, phi):
    log_total, w = ORIG["det_shares"](sys, phi)
    return log_total, w * np.exp(log_total - np.max(log_total))


def _green_first_determinant(sys, phi):
    if sys.dets is None:
        return ORIG["green"](sys, phi)
    return afqmc.det_green(sys, sys.dets[0], phi)


def _energy_from_mixed_green(sys, phi, chunk=0):
    if sys.dets is None:
        return ORIG["local_energy"](sys, phi, chunk)
    return afqmc.energy_from_green(sys, afqmc.green(sys, phi))


def _energy_abs_shares(sys, phi, chunk=0):
    if sys.dets is None:
        return ORIG["local_energy"](sys, phi, chunk)
    _, w = afqmc.det_shares(sys, phi)
    return sum(np.abs(wd) * afqmc.energy_from_green(sys, afqmc.det_green(sys, D, phi))
               for D, wd in zip(sys.dets, w))


MUTANTS = {
    "coefficients squared": ("det_shares", _shares(lambda c: c * c)),
    "coefficients dropped": ("det_shares", _shares(lambda c: np.ones_like(c))),
    "shares not normalised": ("det_shares", _shares_unnormalised),
    "G of the first determinant only": ("green", _green_first_determinant),
    "E_L from the mixed G": ("local_energy", _energy_from_mixed_green),
    "E_L with |w_d|": ("local_energy", _energy_abs_shares),
    "overlap of conj(Phi) per determinant":
        ("det_overlap", lambda s, D, phi: ORIG["det_overlap"](s, D, np.conj(phi))),
}


def first_failing_pin():
    for name, pin in PINS:
        try:
            pin()
        except Exception:
            return name
    return None


def test_control_passes_every_pin():
    assert first_failing_pin() is None


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(monkeypatch, mutant):
    target, fn = MUTANTS[mutant]
    monkeypatch.setattr(afqmc, target, fn)
    assert first_failing_pin() is not None, f"no pin catches: {mutant}"
