"""Whole-algorithm pins of the oracle on the FCI-sized synthetic pair (M=8, Nchol=24).

* Free projection is exact up to Trotter error (Sec. II.A): its mixed energy at
  imaginary time tau must match <psi_T|H e^{-tau H}|psi_T>/<psi_T|e^{-tau H}|psi_T>
  from the dense Hamiltonian within the statistical error.
* Identical systems with shared fields give Delta E = 0 exactly at every
  measurement (perfect walker-pair correlation, Sec. III.C).
* Sharing the fields lowers the standard error of Delta E (Sec. II.B, Fig. 1).
"""
import numpy as np
import pytest

from oracle import afqmc, fci, stats
from synthetic import CONFIGS, build_system


def c1(which, dt, mode=afqmc.PHASELESS):
    d = build_system(**CONFIGS["C1"][which])
    return afqmc.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt, mode=mode), d


@pytest.mark.parametrize("which", ["A", "B"])
def test_free_projection_matches_exact_projection(which):
    dt = 0.01
    s, d = c1(which, dt, mode=afqmc.FREE)
    H = fci.hamiltonian(d["h1"], d["L"], d["n_up"], d["n_dn"])
    psi = fci.determinant_vector(d["trial"], d["n_up"], d["n_dn"])
    r = afqmc.run_pair(s, None, 4096, 40, seed=11, energy_every=20, mgs_every=5, n_repeats=16)
    m, se = stats.per_tau(r["E"][0])
    taus = np.array(r["steps"]) * dt
    exact = fci.projected_energy(H, psi, taus)
    assert np.all(np.abs(m - exact) < 3 * se), (m, exact, se)
    # the projection really moved the energy away from E_HF by many error bars
    assert np.all(np.abs(exact - s.E_T) > 10 * se)


def test_free_projection_one_electron():
    from synthetic import make_hamiltonian
    M, dt = 4, 0.02
    h1, L = make_hamiltonian(M, 3, 21)
    trial = np.linalg.eigh(h1)[1][:, 1:2]          # deliberately not the ground orbital
    trial = trial + 0.5 * np.linalg.eigh(h1)[1][:, 0:1]
    trial /= np.linalg.norm(trial)
    s = afqmc.System(h1, L, trial, 1, 0, dt, mode=afqmc.FREE)
    r = afqmc.run_pair(s, None, 2048, 100, seed=2, energy_every=25, n_repeats=16)
    m, se = stats.per_tau(r["E"][0])
    H = fci.hamiltonian(h1, L, 1, 0)
    np.testing.assert_allclose(H, h1, atol=1e-14)          # one electron: H = h1
    exact = fci.projected_energy(H, trial[:, 0], np.array(r["steps"]) * dt)
    assert np.all(np.abs(m - exact) < 3 * se + 1e-12), (m, exact, se)


def test_identical_systems_give_exactly_zero_difference():
    s, _ = c1("A", 0.01)
    s2, _ = c1("A", 0.01)
    r = afqmc.run_pair(s, s2, 24, 40, seed=3, n_repeats=3)
    assert np.array_equal(r["E"][0], r["E"][1])


def test_correlated_sampling_reduces_error_of_difference():
    """Same basis, same electrons, one-body part changed (the ghost-basis case of Sec. II.C):
    V and v are identical, only T differs, and sharing the fields must cut the error of
    Delta E by a large factor relative to independent fields (11 repeats x 12 walkers,
    the protocol of Fig. 1)."""
    from synthetic.scf import scf_trial
    d = build_system(**CONFIGS["C1"]["A"])
    rng = np.random.default_rng(5)
    h1b = d["h1"] + np.diag(0.1 * rng.standard_normal(d["M"]))
    tb, _, _ = scf_trial(h1b, d["L"], 2, 2)
    sA = afqmc.System(d["h1"], d["L"], d["trial"], 2, 2, 0.01)
    sB = afqmc.System(h1b, d["L"], tb, 2, 2, 0.01)
    R, nw_per = 11, 12
    nw = R * nw_per
    corr = afqmc.run_pair(sA, sB, nw, 100, seed=4, n_repeats=R)
    dc = corr["E"][1] - corr["E"][0]
    ub = afqmc.run_pair(sB, None, nw, 100, seed=10_004, n_repeats=R)
    du = ub["E"][0] - corr["E"][0]
    taus = np.array(corr["steps"]) * 0.01
    _, se_c = stats.per_tau(dc)
    _, se_u = stats.per_tau(du)
    assert np.mean(se_c) < 0.2 * np.mean(se_u)
    mc, sc, _ = stats.delta_e_estimate(dc, taus, 0.3)
    mu, su, _ = stats.delta_e_estimate(du, taus, 0.3)
    assert sc < 0.2 * su
    assert abs(mc - mu) < 3 * np.hypot(sc, su)     # same difference, smaller error


def test_seed_B_draws_independent_fields_for_B_only():
    """run_pair(seed_B=...) is the uncorrelated comparison: A follows its solo run on the
    common key and B its solo run on its own key, bit for bit."""
    sA, _ = c1("A", 0.01)
    sB, _ = c1("B", 0.01)
    nw, R, steps = 8, 2, 15
    ind = afqmc.run_pair(sA, sB, nw, steps, seed=7, seed_B=8, n_repeats=R)
    soloA = afqmc.run_pair(sA, None, nw, steps, seed=7, n_repeats=R)
    soloB = afqmc.run_pair(sB, None, nw, steps, seed=8, n_repeats=R)
    assert np.array_equal(ind["E"][0], soloA["E"][0])
    assert np.array_equal(ind["E"][1], soloB["E"][0])
    same = afqmc.run_pair(sA, sB, nw, steps, seed=7, n_repeats=R)
    assert np.array_equal(same["E"][0], ind["E"][0])
    assert not np.array_equal(same["E"][1], ind["E"][1])


def test_dead_walker_with_non_finite_energy_does_not_reach_the_estimate():
    """A walker killed for a non-finite overlap keeps a non-finite determinant; with w = 0 it
    must add nothing to the mixed estimate (Sec. II.B: dead walkers no longer contribute)."""
    s, _ = c1("A", 0.01)
    w = np.array([0.7, 0.0, 1.3, 0.9], dtype=complex)
    eloc = np.array([-8.1, np.nan, -8.3, -8.2], dtype=complex)
    groups = np.zeros(4, int)
    E, W = afqmc.mixed_energy(s, w, eloc, groups, 1)
    live = w != 0
    assert np.isfinite(E[0]) and W[0] == w.real.sum()
    assert abs(E[0] - np.sum(w[live].real * eloc[live].real) / W[0]) < 1e-15
