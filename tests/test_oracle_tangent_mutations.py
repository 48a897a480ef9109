"""Planted mistakes in the oracle's tangent mode, each of which must fail a pin.

A mutant is the source of oracle/tangent.py with one slip written in: a dropped term of a
product rule, a missing projection, a sign, a wrong factor, a skipped transformation after
Gram-Schmidt. The pins of test_oracle_tangent.py run against the compiled copy: central
differences of whole runs under common fields (with and without an active force-bias cap),
and the exact derivative at the trial. The unmutated source must pass them all.

Not listed, because no measurement can see it: dropping the dt dE_T term of d log I. It adds
the same constant to every walker's d log w, and a factor common to all weights cancels in
sum w E_L / sum w.
"""
import pytest

import test_oracle_tangent as PT
from mutation_util import compile_variant, mutate, oracle_source

SRC = oracle_source("tangent.py")

MUTANTS = {
    "dTheta without -Theta dO": ("dTheta = (dphi[:, :, a:b] - Theta @ dO) @ Oi",
                                 "dTheta = dphi[:, :, a:b] @ Oi"),
    "d log O as elementwise sum": ('dlogO += np.einsum("wab,wba->w", Oi, dO)',
                                   'dlogO += np.einsum("wab,wab->w", Oi, dO)'),
    "cap derivative without projection": (
        "dcap = sys.fb_cap * (draw / safe - raw * np.real(np.conj(raw) * draw) / safe ** 3)",
        "dcap = sys.fb_cap * (draw / safe)"),
    "Taylor product rule without A dT": ("T, dT = (A @ T) / n, (dA @ T + A @ dT) / n",
                                         "T, dT = (A @ T) / n, (dA @ T) / n"),
    "second half step without dE": ("dphi3 = dE @ phi2 + E @ dphi2", "dphi3 = E @ dphi2"),
    "x.xbar derivative with x for x - xbar": ("np.sum((xs - xbar) * dxbar, axis=1)",
                                              "np.sum(xs * dxbar, axis=1)"),
    "cos-cut derivative sign": ("tw.dlogw[idx] + dlogI.real - tanv * dlogR.imag",
                                "tw.dlogw[idx] + dlogI.real + tanv * dlogR.imag"),
    "tangent not transformed by MGS": (
        "dphi[:, :, a:b] = dphi[:, :, a:b] @ np.linalg.inv(np.triu(R))",
        "dphi[:, :, a:b] = dphi[:, :, a:b]"),
    "exchange derivative without 2": ('dex = dex + 2 * np.einsum("wgik,wgki->wg", LG, LdG)',
                                      'dex = dex + np.einsum("wgik,wgki->wg", LG, LdG)'),
    "direct one-body term dropped": ('de1 = sum(np.einsum("ij,wji->w", ts.P, Gs) + ',
                                     'de1 = sum(0 * np.einsum("ij,wji->w", ts.P, Gs) + '),
    "weight normalisation derivative dropped": (
        "dE = (np.sum(dw * eloc.real + w * deloc.real) - E * np.sum(dw)) / W",
        "dE = np.sum(dw * eloc.real + w * deloc.real) / W"),
    "half-step factor of dE": ("_, self.dE = frechet_exp(B, -0.5 * sys.dt * self.P)",
                               "_, self.dE = frechet_exp(B, -sys.dt * self.P)"),
}

PINS = [
    ("trial-state derivative", PT.test_tangent_of_trial_energy_and_one_body_term),
    ("central differences, A", lambda: PT.test_tangent_matches_central_differences("A", 1.0)),
    ("central differences, B", lambda: PT.test_tangent_matches_central_differences("B", 1.0)),
    ("central differences, cap active",
     lambda: PT.test_tangent_matches_central_differences("A", 0.05)),
]


def first_failing_pin(monkeypatch, mod):
    monkeypatch.setattr(PT, "tangent", mod)
    for name, pin in PINS:
        try:
            pin()
        except Exception:
            return name
    return None


def test_unmutated_source_passes_every_pin(monkeypatch):
    assert first_failing_pin(monkeypatch, compile_variant(SRC, "tangent_control")) is None


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(monkeypatch, mutant):
    old, new = MUTANTS[mutant]
    mod = mutate(SRC, old, new, "tangent_mutant")
    assert first_failing_pin(monkeypatch, mod) is not None, f"no pin catches: {mutant}"
