"""Pins of the oracle's preliminary equilibration scheme (Sec. II.C): the comb's closed-form
properties, and the seeding of the secondary system checked in the many-body space (the
state the weighted walkers represent is unchanged by the change of trial)."""
import numpy as np
import pytest

from oracle import afqmc, fci, pes
from synthetic import CONFIGS, build_system, make_hamiltonian, scf_trial


def test_comb_keeps_the_total_weight_and_skips_dead_walkers():
    rng = np.random.default_rng(1)
    w = rng.exponential(size=40)
    w[[0, 3, 4, 17, 39]] = 0.0        # a leading dead walker: at u = 0 the first point is 0
    for u in (0.0, 0.25, 0.999999):
        pick, w_new = pes.comb_select(w, w.size, u)
        assert abs(w_new * w.size - w.sum()) < 1e-12 * w.sum()
        assert np.all(w[pick] > 0)
        assert np.all(np.diff(pick) >= 0)


def test_comb_expected_copies_are_the_weight_shares():
    """Averaged over u in [0, 1), walker k is chosen n w_k / W times (exactly, for the comb);
    a midpoint grid of K values of u reproduces that to 2 / K."""
    rng = np.random.default_rng(2)
    w = rng.exponential(size=25)
    w[7] = 0.0
    n, K = 30, 4000
    counts = np.zeros(w.size)
    for u in (np.arange(K) + 0.5) / K:
        pick, _ = pes.comb_select(w, n, u)
        counts += np.bincount(pick, minlength=w.size)
    np.testing.assert_allclose(counts / K, n * w / w.sum(), rtol=0, atol=2.0 / K + 1e-12)


def test_comb_of_equal_weights_keeps_every_walker():
    """Equal weights: point j lies inside walker j's share. (At u = 0 the points fall on the
    shares' boundaries, where the rounding of the running sum decides; u there is a set of
    measure zero, so it is left out.)"""
    for u in (0.25, 0.5, 0.999):
        pick, w_new = pes.comb_select(np.full(9, 0.3), 9, u)
        assert np.array_equal(pick, np.arange(9)) and abs(w_new - 0.3) < 1e-15


def test_population_control_stays_within_each_repeat():
    d = build_system(**CONFIGS["C1"]["A"])
    s = afqmc.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], 0.01)
    nw, R = 24, 3
    wk = afqmc.Walkers(s, nw)
    rng = np.random.default_rng(3)
    for t in range(5):
        afqmc.propagate(s, wk, rng.standard_normal((nw, s.X)))
    wk.w[5] = 0.0
    wk.alive[5] = False
    groups = afqmc.repeat_groups(nw, R)
    before = wk.copy()
    pes.population_control(s, wk, groups, R, np.array([0.1, 0.6, 0.9]))
    for r in range(R):
        m = groups == r
        assert abs(wk.w[m].real.sum() - before.w[m].real.sum()) < 1e-12 * before.w[m].real.sum()
        assert np.allclose(wk.w[m].real, wk.w[m].real[0]) and np.all(wk.alive[m])
        mine = before.phi[m]
        for k in np.nonzero(m)[0]:       # every new walker is a copy of one of the same repeat
            assert any(np.array_equal(wk.phi[k], p) for p in mine)
    assert not any(np.array_equal(wk.phi[k], before.phi[5]) for k in range(nw))


def _walkers_near(trial, n, seed, scale=0.15):
    rng = np.random.default_rng(seed)
    return trial[None] + scale * rng.standard_normal((n,) + trial.shape)


def _represented_state(phi, w, psi_vec, n_up, n_dn):
    """sum_k w_k |phi_k> / <psi|phi_k> in the many-body space (FCI-space overlaps)."""
    out = 0
    for p, wk in zip(phi, w):
        v = fci.determinant_vector(p, n_up, n_dn)
        out = out + wk * v / (psi_vec @ v)
    return out


@pytest.mark.parametrize("n_dn_B", [2, 1])
def test_seeding_keeps_the_represented_state(n_dn_B):
    """The secondary walkers with weights w_A R represent, with B's trial, what the primary
    walkers represent with A's trial (same electrons), or the same with the last spin-down
    trial orbital removed (an ion); real positive ratios, so no phase is projected."""
    M, X, n_up, n_dn = 5, 4, 2, 2
    h1, L = make_hamiltonian(M, X, 8)
    tA, _, _ = scf_trial(h1, L, n_up, n_dn)
    sA = afqmc.System(h1, L, tA, n_up, n_dn, 0.01)
    # B's trial: A's orbitals mixed by a small rotation inside each spin block (same space
    # for n_dn_B = 2, so the overlaps stay real and positive), or the ion's HF orbitals
    if n_dn_B == n_dn:
        rot = np.linalg.qr(np.eye(M) + 0.2 * np.random.default_rng(4).standard_normal((M, M)))[0]
        tB = rot @ tA
        tB /= np.sign(np.diag(tA.T @ tB))[None, :]
    else:
        tB, _, _ = scf_trial(h1, L, n_up, n_dn_B)
    sB = afqmc.System(h1, L, tB, n_up, n_dn_B, 0.01)
    phi = _walkers_near(tA, 6, seed=5)
    w = np.random.default_rng(6).exponential(size=6).astype(complex)
    wkA = afqmc.Walkers(sA, 6, phi=phi, w=w)
    wkB = pes.seed_secondary(sA, sB, wkA)
    assert np.array_equal(wkB.phi, phi[:, :, pes.seed_columns(sA, sB)])
    psiA = fci.determinant_vector(tA, n_up, n_dn)
    psiB = fci.determinant_vector(tB, n_up, n_dn_B)
    ovA = np.array([psiA @ fci.determinant_vector(p, n_up, n_dn) for p in phi])
    ovB = np.array([psiB @ fci.determinant_vector(p, n_up, n_dn_B) for p in wkB.phi])
    assert np.all((ovB / ovA).real > 0) and np.allclose((ovB / ovA).imag, 0)
    lhs = _represented_state(wkB.phi, wkB.w, psiB, n_up, n_dn_B)
    # the primary walkers' (truncated) determinants weighted as with A's trial
    rhs = sum(wk_ * fci.determinant_vector(p, n_up, n_dn_B) / oa
              for p, wk_, oa in zip(wkB.phi, w, ovA))
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-12 * np.abs(rhs).max())


def test_seeding_projects_the_phase_of_the_ratio():
    """One trial column negated flips every overlap: R = -1, the walker gets weight 0 (cos
    cut). Two negated columns in one spin block leave R = +1 and the weight unchanged."""
    d = build_system(**CONFIGS["C1"]["A"])
    sA = afqmc.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], 0.01)
    wkA = afqmc.Walkers(sA, 5, phi=_walkers_near(d["trial"], 5, seed=7).astype(complex),
                        w=np.full(5, 0.7 + 0j))
    for cols, alive in (([0], False), ([0, 1], True)):
        tB = d["trial"].copy()
        tB[:, cols] *= -1
        sB = afqmc.System(d["h1"], d["L"], tB, d["n_up"], d["n_dn"], 0.01)
        wkB = pes.seed_secondary(sA, sB, wkA)
        assert np.all(wkB.alive == alive)
        np.testing.assert_allclose(wkB.w.real, 0.7 if alive else 0.0, rtol=1e-12, atol=0)


def test_pes_with_identical_systems_gives_zero_difference_and_continues_the_stream():
    d = build_system(**CONFIGS["C1"]["A"])
    mk = lambda: afqmc.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], 0.01)
    sA, sB = mk(), mk()
    nw, R, n_eq, n_steps, seed = 12, 2, 10, 10, 9
    u = np.array([[0.3, 0.8], [0.55, 0.05]])
    r = pes.run_pes(sA, sB, nw, n_eq, n_steps, seed, u, n_repeats=R)
    assert np.array_equal(r["E"][0], r["E"][1])
    # A alone: the same equilibration and combs by hand, then its continuation at step n_eq
    from oracle.philox import gaussian_fields
    wk = afqmc.Walkers(sA, nw)
    groups = afqmc.repeat_groups(nw, R)
    for t in range(n_eq):
        afqmc.propagate(sA, wk, gaussian_fields(seed, t, np.arange(nw), sA.X))
        if (t + 1) % 5 == 0:
            afqmc.orthonormalise(sA, wk)
            pes.population_control(sA, wk, groups, R, u[(t + 1) // 5 - 1])
    solo = afqmc.run_pair(sA, None, nw, n_steps, seed, n_repeats=R, walkers=(wk,), t0=n_eq)
    assert np.array_equal(solo["E"][0], r["E"][0])


def test_secondary_with_more_electrons_is_refused():
    d = build_system(**CONFIGS["C1"]["B"])     # 2/1
    sA = afqmc.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], 0.01)
    dB = build_system(**CONFIGS["C1"]["A"])    # 2/2
    sB = afqmc.System(dB["h1"], dB["L"], dB["trial"], dB["n_up"], dB["n_dn"], 0.01)
    with pytest.raises(ValueError):
        pes.seed_columns(sA, sB)
