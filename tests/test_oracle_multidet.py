"""Pins of the oracle's multi-determinant trial (Sec. II.D; the truncated CASSCF trials of
Sec. III) against the many-body space: none of them re-types the oracle's per-determinant sums.

* <psi_T|phi> is the contraction of the trial's many-body vector with the walker's;
* G is the derivative of log <psi_T|e^{e E}|phi> (Thouless), rhobar the derivative along L_g;
* E_L is <psi_T|H|phi> / <psi_T|phi> with the dense H of Eq. 1;
* with the exact ground state as trial, E_L is E_0 for any walker (zero variance);
* one determinant with coefficient 1 is the single-determinant oracle (up to rounding);
* free projection with the multi-determinant trial still converges to the exact projection.
"""
import itertools

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import afqmc, fci, stats
from synthetic import CONFIGS, build_system, make_hamiltonian, scf_trial
from synthetic.multidet import cas_trial


def many_body(dets, coeffs, n_up, n_dn):
    return sum(c * fci.determinant_vector(D, n_up, n_dn) for D, c in zip(dets, coeffs))


def md_system(M=6, X=7, n_up=2, n_dn=2, seed=13, n_orb=5, dt=0.01, mode=afqmc.PHASELESS):
    h1, L = make_hamiltonian(M, X, seed)
    trial, _, _ = scf_trial(h1, L, n_up, n_dn)
    dets, c, start, _ = cas_trial(h1, L, trial, n_up, n_dn, n_orb, threshold=0.02)
    s = afqmc.System(h1, L, None, n_up, n_dn, dt, mode=mode, dets=dets, coeffs=c, start=start)
    return s, dets, c


def random_phi(M, N, n=1, seed=3):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, M, N)) + 1j * rng.standard_normal((n, M, N))


OCC = [(2, 2), (2, 1), (3, 1)]


@pytest.mark.parametrize("n_up,n_dn", OCC)
def test_overlap_is_many_body_overlap(n_up, n_dn):
    s, dets, c = md_system(n_up=n_up, n_dn=n_dn)
    assert len(c) >= 3
    psi = many_body(dets, c, n_up, n_dn)
    phi = random_phi(s.M, s.N, 3)
    for k in range(3):
        want = psi @ fci.determinant_vector(phi[k], n_up, n_dn)
        got = np.exp(afqmc.overlap(s, phi[k:k + 1])[0])
        assert abs(got - want) < 1e-12 * abs(want)


@pytest.mark.parametrize("n_up,n_dn", OCC)
def test_green_function_is_log_overlap_derivative(n_up, n_dn):
    s, _, _ = md_system(n_up=n_up, n_dn=n_dn)
    phi = random_phi(s.M, s.N, 1, seed=5)
    G = afqmc.green(s, phi)
    E = np.random.default_rng(8).standard_normal((s.M, s.M))
    eps = 1e-5
    for si, (a, b) in enumerate(s.spins):
        if b == a:
            continue

        def logov(e):
            p = phi.copy()
            p[0][:, a:b] = expm(e * E) @ p[0][:, a:b]
            return afqmc.overlap(s, p)[0]

        fd = (logov(eps) - logov(-eps)) / (2 * eps)
        assert abs(fd - np.sum(E * G[si][0])) < 1e-7 * max(1, abs(fd))


def test_force_bias_is_log_overlap_derivative():
    s, _, _ = md_system(n_up=2, n_dn=1)
    phi = random_phi(s.M, s.N, 1, seed=6)
    rb = afqmc.rhobar(s, afqmc.green(s, phi))[0]
    eps = 1e-5
    for g in range(s.X):
        lo = [afqmc.overlap(s, (expm(e * s.L[g]) @ phi[0])[None])[0] for e in (eps, -eps)]
        fd = (lo[0] - lo[1]) / (2 * eps)
        assert abs(fd - rb[g]) < 1e-7 * max(1, abs(rb[g]))


@pytest.mark.parametrize("n_up,n_dn", OCC)
def test_local_energy_is_many_body_mixed_estimate(n_up, n_dn):
    s, dets, c = md_system(n_up=n_up, n_dn=n_dn)
    H = fci.hamiltonian(s.h1, s.L, n_up, n_dn)
    psi = many_body(dets, c, n_up, n_dn)
    phi = random_phi(s.M, s.N, 4, seed=9)
    el = afqmc.local_energy(s, phi)
    for k in range(4):
        v = fci.determinant_vector(phi[k], n_up, n_dn)
        want = (psi @ H @ v) / (psi @ v)
        assert abs(el[k] - want) < 1e-10 * abs(want)


def test_exact_ground_state_trial_has_zero_variance_local_energy():
    """Every determinant of the basis, with the FCI ground state's coefficients: H psi_T = E_0
    psi_T, so <psi_T|H|phi> = E_0 <psi_T|phi> for any walker."""
    M, n_up, n_dn = 5, 2, 2
    h1, L = make_hamiltonian(M, 6, 17)
    H = fci.hamiltonian(h1, L, n_up, n_dn)
    e0, ci = fci.ground_state(H)
    I = np.eye(M)
    dets = [np.concatenate([I[:, list(u)], I[:, list(d)]], axis=1)
            for u in itertools.combinations(range(M), n_up)
            for d in itertools.combinations(range(M), n_dn)]
    start = np.linalg.eigh(h1)[1][:, [0, 1, 0, 1]]
    s = afqmc.System(h1, L, None, n_up, n_dn, 0.01, dets=np.array(dets), coeffs=ci, start=start)
    phi = random_phi(M, n_up + n_dn, 5, seed=12)
    el = afqmc.local_energy(s, phi)
    assert np.max(np.abs(el - e0)) < 1e-9 * abs(e0)


def test_one_determinant_is_the_single_determinant_oracle():
    """Up to rounding: the sum over determinants is formed relative to the largest overlap."""
    d = build_system(**CONFIGS["C1"]["B"])
    one = afqmc.System(d["h1"], d["L"], d["trial"], 2, 1, 0.01)
    md = afqmc.System(d["h1"], d["L"], None, 2, 1, 0.01, dets=d["trial"][None], coeffs=[1.0])
    ra = afqmc.run_pair(one, None, 16, 20, seed=3, n_repeats=2)
    rb = afqmc.run_pair(md, None, 16, 20, seed=3, n_repeats=2)
    np.testing.assert_allclose(rb["E"][0], ra["E"][0], rtol=1e-12)
    np.testing.assert_allclose(rb["walkers"][0].phi, ra["walkers"][0].phi, rtol=0, atol=1e-12)


def test_background_and_energy_shift_follow_the_first_determinant():
    """Reading: <rho_g>_T, K and E_T of a multi-determinant trial are those of D_0."""
    s, dets, _ = md_system()
    ref = afqmc.System(s.h1, s.L, dets[0], s.n_up, s.n_dn, s.dt)
    assert np.array_equal(s.rho_mf, ref.rho_mf) and s.E_T == ref.E_T
    assert np.array_equal(s.expK, ref.expK)
    # the walkers' start overlaps every determinant of the expansion
    logO = [afqmc.det_overlap(s, D, s.start[None].astype(complex))[0] for D in dets]
    assert min(np.exp(np.real(logO))) > 1e-4


def test_free_projection_with_multideterminant_trial_matches_exact_projection():
    """Free projection is exact for any trial (Sec. II.A): with the truncated CASCI trial and
    walkers started outside it, E(tau) follows <psi_T|H e^{-tau H}|phi_0> / <psi_T|e^{-tau H}|phi_0>."""
    d = build_system(**CONFIGS["C1"]["A"])
    dets, c, start, _ = cas_trial(d["h1"], d["L"], d["trial"], 2, 2, 6, threshold=0.05)
    dt = 0.01
    s = afqmc.System(d["h1"], d["L"], None, 2, 2, dt, mode=afqmc.FREE, dets=dets, coeffs=c,
                     start=start)
    r = afqmc.run_pair(s, None, 2048, 40, seed=11, energy_every=20, mgs_every=5, n_repeats=16)
    m, se = stats.per_tau(r["E"][0])
    H = fci.hamiltonian(d["h1"], d["L"], 2, 2)
    psi = many_body(dets, c, 2, 2)
    v0 = fci.determinant_vector(start, 2, 2)
    lam, U = np.linalg.eigh(H)
    a, b = U.T @ psi, U.T @ v0
    exact = [np.sum(a * b * lam * np.exp(-t * lam)) / np.sum(a * b * np.exp(-t * lam))
             for t in np.array(r["steps"]) * dt]
    assert np.all(np.abs(m - exact) < 3 * se + 1e-12), (m, exact, se)
