"""Planted mistakes in the oracle's reverse pass, each of which must fail a pin.

A mutant is the source of oracle/adjoint.py with one slip written in (a missing complex
conjugate, A where A^H belongs, a sign, a dropped term or factor, a skipped cap projection).
It is compiled as a separate module inside the oracle package and the adjoint pins of
test_oracle_adjoint.py run against it: the gradient contracted with symmetric P against the
tangent mode (itself pinned by central differences of whole runs), and one entry against a
central difference. The unmutated source must pass them all. Slips that change only the
antisymmetric part of dE/dh1 are not listed: h1 is symmetric, so no measurement sees them.
"""
import types

import pytest

import test_oracle_adjoint as PA
from mutation_util import compile_variant, mutate, oracle_source

SRC = oracle_source("adjoint.py")

MUTANTS = {
    "cos-cut term sign": ("Rbar = lb * (1.0 - 1j * np.tan(th))",
                          "Rbar = lb * (1.0 + 1j * np.tan(th))"),
    "x.xbar adjoint without conj": ("xbb = lb[:, None] * np.conj(xs - xb)",
                                    "xbb = lb[:, None] * (xs - xb)"),
    "Taylor Abar without conj": ("Abar += Tb @ np.conj(np.swapaxes(terms[n - 1], 1, 2)) / n",
                                 "Abar += Tb @ np.swapaxes(terms[n - 1], 1, 2) / n"),
    "Taylor adjoint with A for A^H": ("Tb = pb2 + (AH @ Tb) / n", "Tb = pb2 + (A @ Tb) / n"),
    "O^{-1} term of G dropped": ("phibar[:, :, a:b] += Psi[None] @ Ob",
                                 "phibar[:, :, a:b] += 0.0 * (Psi[None] @ Ob)"),
    "MGS adjoint without conj": ("pb[:, :, a:b] @ np.conj(np.swapaxes(np.linalg.inv(R), 1, 2))",
                                 "pb[:, :, a:b] @ np.swapaxes(np.linalg.inv(R), 1, 2)"),
    "one-body half step factor": ("h1bar += -0.5 * sys.dt * LE", "h1bar += -sys.dt * LE"),
    "cap projection skipped": ("(sys.fb_cap / safe) * (xbb - np.real(np.conj(xbb) * xr) * xr / safe ** 2)",
                               "(sys.fb_cap / safe) * xbb"),
    "mean-field scalar adjoint without conj": (
        "cbar = Rbar[:, None] * np.conj(-1j * sys.sqrt_dt * sys.rho_mf)[None, :]",
        "cbar = Rbar[:, None] * (-1j * sys.sqrt_dt * sys.rho_mf)[None, :]"),
    "exchange sign in dE_L/dG": ('F = sys.h1[None] + np.einsum("wg,gij->wij", rb, sys.L) - LGL',
                                 'F = sys.h1[None] + np.einsum("wg,gij->wij", rb, sys.L) + LGL'),
}

PINS = [
    ("contraction with P, A", lambda: PA.test_gradient_contracts_to_tangent("A", 1.0)),
    ("contraction with P, B", lambda: PA.test_gradient_contracts_to_tangent("B", 1.0)),
    ("contraction with P, cap active", lambda: PA.test_gradient_contracts_to_tangent("A", 0.05)),
    ("central difference", PA.test_gradient_entry_by_central_differences),
]


def first_failing_pin(monkeypatch, mod: types.ModuleType):
    monkeypatch.setattr(PA, "adjoint", mod)
    for name, pin in PINS:
        try:
            pin()
        except Exception:
            return name
    return None


def test_unmutated_source_passes_every_pin(monkeypatch):
    assert first_failing_pin(monkeypatch, compile_variant(SRC, "adjoint_control")) is None


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(monkeypatch, mutant):
    old, new = MUTANTS[mutant]
    mod = mutate(SRC, old, new, "adjoint_mutant")
    assert first_failing_pin(monkeypatch, mod) is not None, f"no pin catches: {mutant}"
