"""The moderate-coupling reading of the synthetic recipe, pinned by the statistic it holds fixed.

The reading: every L_g of the recipe is scaled so that the one-body matrix of one step's fields,
sum_g x_g L_g with x_g ~ N(0, 1), has the same expected spectral norm (2 sqrt 2) on every
workload; at the step dt = 0.005 of the M >= 64 workloads, sqrt(dt) times that norm, the size
of the exponent one step applies to a walker (Eqs. 4-5, 11), is 0.2.  These tests draw the
fields and measure the norm directly (no use of the formula that sets the scale), so a wrong
variance sum, a missing sqrt(M) or a scale applied twice fails them.
"""
import numpy as np
import pytest

from synthetic import CONFIGS, build_system
from synthetic.hamiltonian import STEP_NORM, field_entry_sd, make_hamiltonian, moderate_coupling


def step_norm(L, dt, draws=12, seed=5):
    rng = np.random.default_rng(seed)
    X = L.shape[0]
    return np.sqrt(dt) * np.mean([np.linalg.norm(np.tensordot(rng.standard_normal(X), L, 1), 2)
                                  for _ in range(draws)])


@pytest.mark.parametrize("cfg,which", [("C2", "A"), ("C3", "A"), ("C3", "B"), ("C4", "A"),
                                       ("C4", "B"), ("C5", "A")])
def test_moderate_coupling_holds_the_per_step_norm(cfg, which):
    d = CONFIGS[cfg][which]
    dt = CONFIGS[cfg]["dt"]
    assert dt == 0.005
    _, L = make_hamiltonian(d["M"], d["X"], d["seed"], coupling=moderate_coupling(d["M"], d["X"]))
    nrm = step_norm(L, dt)
    # the semicircle edge 2 sigma sqrt(M) is approached from below at finite M
    assert 0.185 < nrm <= 0.2 * 1.02, nrm
    assert np.sqrt(dt) * STEP_NORM == pytest.approx(0.2)


def test_literal_recipe_steps_are_an_order_larger():
    """Why the reading exists: at M = 64, X = 320 the recipe as stated takes steps of norm ~2."""
    d = CONFIGS["C2"]["A"]
    _, L = make_hamiltonian(d["M"], d["X"], d["seed"], coupling=1.0)
    assert step_norm(L, CONFIGS["C2"]["dt"], draws=4) > 1.5


def test_entry_variance_of_the_field_matrix():
    """Entries of sum_g x_g L_g (coupling 1) have variance 0.09 sum_g exp(-8 g / X)."""
    M, X = 24, 40
    _, L = make_hamiltonian(M, X, 11)
    rng = np.random.default_rng(3)
    A = np.einsum("sg,gij->sij", rng.standard_normal((4000, X)), L)
    emp = A[:, np.triu_indices(M)[0], np.triu_indices(M)[1]].var()
    assert emp == pytest.approx(field_entry_sd(X) ** 2, rel=0.03)


def test_moderate_trials_converge():
    """The trials of the M = 64 and M = 128 pairs come from a converged SCF."""
    for cfg in ("C2", "C3"):
        for which in ("A", "B"):
            s = build_system(**dict(CONFIGS[cfg][which], coupling="moderate"))
            assert s["scf_converged"], (cfg, which)
