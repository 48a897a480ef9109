"""Pins of the oracle against brute force, closed forms and invariants.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
sign, a transposed operand, a missing factor i or 1/2) fails at least one of
them; none of them re-types the oracle's own formula.
"""
import numpy as np
import pytest
from scipy.linalg import expm

from oracle import afqmc, fci
from synthetic import make_hamiltonian, scf_trial
from synthetic.scf import hf_energy


def small_system(M=5, X=6, n_up=2, n_dn=2, seed=11, dt=0.01, mode=afqmc.PHASELESS,
                 taylor_order=6, fb_cap=1.0, scale=1.0):
    h1, L = make_hamiltonian(M, X, seed)
    L = L * scale
    trial, ok, _ = scf_trial(h1, L, n_up, n_dn)
    return afqmc.System(h1, L, trial, n_up, n_dn, dt, fb_cap=fb_cap, mode=mode,
                        taylor_order=taylor_order)


def random_phi(M, N, n=1, seed=3):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, M, N)) + 1j * rng.standard_normal((n, M, N))


OCC = [(2, 2), (2, 1), (3, 1), (1, 0)]


@pytest.mark.parametrize("n_up,n_dn", OCC)
def test_overlap_is_many_body_overlap(n_up, n_dn):
    s = small_system(n_up=n_up, n_dn=n_dn)
    phi = random_phi(s.M, s.N, 3)
    psi = fci.determinant_vector(s.trial, n_up, n_dn)
    for k in range(3):
        v = fci.determinant_vector(phi[k], n_up, n_dn)
        want = psi @ v
        got = np.exp(afqmc.overlap(s, phi[k:k + 1])[0])
        assert abs(got - want) < 1e-12 * abs(want)


@pytest.mark.parametrize("n_up,n_dn", OCC)
def test_green_function_is_log_overlap_derivative(n_up, n_dn):
    """d/de log <psi_T| e^{e E} |phi> at 0 equals sum_ij E_ij G_ij (spin-resolved)."""
    s = small_system(n_up=n_up, n_dn=n_dn)
    phi = random_phi(s.M, s.N, 1, seed=5)
    G = afqmc.green(s, phi)
    rng = np.random.default_rng(8)
    E = rng.standard_normal((s.M, s.M))
    eps = 1e-5
    for si, (a, b) in enumerate(s.spins):
        if b == a:
            continue

        def logov(e):
            p = phi.copy()
            p[0][:, a:b] = expm(e * E) @ p[0][:, a:b]
            return afqmc.overlap(s, p)[0]

        fd = (logov(eps) - logov(-eps)) / (2 * eps)
        want = np.sum(E * G[si][0])
        assert abs(fd - want) < 1e-7 * max(1, abs(want))


def test_force_bias_is_log_overlap_derivative():
    """rhobar_g = d/de log <psi_T| e^{e rho_g} |phi>, summed over spins (Eq. 9 ingredient)."""
    s = small_system(n_up=2, n_dn=1)
    phi = random_phi(s.M, s.N, 1, seed=6)
    rb = afqmc.rhobar(s, afqmc.green(s, phi))[0]
    eps = 1e-5
    for g in range(s.X):
        U = [expm(e * s.L[g]) for e in (eps, -eps)]
        lo = [afqmc.overlap(s, (u @ phi[0])[None])[0] for u in U]
        fd = (lo[0] - lo[1]) / (2 * eps)
        assert abs(fd - rb[g]) < 1e-7 * max(1, abs(rb[g]))


def test_green_function_invariants():
    s = small_system(n_up=3, n_dn=1)
    G = afqmc.green(s, random_phi(s.M, s.N, 2, seed=9))
    for Gs, n in zip(G, (3, 1)):
        for k in range(2):
            assert abs(np.trace(Gs[k]) - n) < 1e-12
            np.testing.assert_allclose(Gs[k] @ Gs[k], Gs[k], atol=1e-11)


@pytest.mark.parametrize("M,n_up,n_dn", [(3, 1, 1), (3, 2, 1), (4, 1, 1)])
def test_fci_two_body_matches_direct_operator_products(M, n_up, n_dn):
    _, L = make_hamiltonian(M, 3, 4)
    V = np.einsum("gik,gjl->ijkl", L, L)
    H = fci.hamiltonian(np.zeros((M, M)), L, n_up, n_dn)
    D = fci.two_body_direct(V, M, n_up, n_dn)
    np.testing.assert_allclose(H, D, atol=1e-13)


@pytest.mark.parametrize("n_up,n_dn", OCC)
def test_local_energy_is_mixed_estimate_in_fci_space(n_up, n_dn):
    """E_L(phi) = <psi_T|H|phi>/<psi_T|phi> with the dense H of Eq. 1 (complex phi)."""
    s = small_system(n_up=n_up, n_dn=n_dn)
    H = fci.hamiltonian(s.h1, s.L, n_up, n_dn)
    psi = fci.determinant_vector(s.trial, n_up, n_dn)
    phi = random_phi(s.M, s.N, 3, seed=21)
    el = afqmc.local_energy(s, phi)
    for k in range(3):
        v = fci.determinant_vector(phi[k], n_up, n_dn)
        want = (psi @ H @ v) / (psi @ v)
        assert abs(el[k] - want) < 1e-11 * abs(want)


@pytest.mark.parametrize("n_up,n_dn", [(2, 2), (2, 1), (3, 0)])
def test_trial_energy_is_hartree_fock_energy(n_up, n_dn):
    s = small_system(n_up=n_up, n_dn=n_dn)
    e_scf = hf_energy(s.h1, s.L, s.trial[:, :n_up], s.trial[:, n_up:])
    H = fci.hamiltonian(s.h1, s.L, n_up, n_dn)
    psi = fci.determinant_vector(s.trial, n_up, n_dn)
    e_fci = psi @ H @ psi / (psi @ psi)
    assert abs(s.E_T - e_scf) < 1e-12 * abs(e_scf)
    assert abs(s.E_T - e_fci) < 1e-12 * abs(e_fci)


def test_one_electron_has_no_two_body_energy():
    """For a single electron the Coulomb and exchange terms of E_L cancel exactly."""
    s = small_system(n_up=1, n_dn=0)
    phi = random_phi(s.M, s.N, 4, seed=2)
    G = afqmc.green(s, phi)
    e1 = np.einsum("ij,wji->w", s.h1, G[0])
    np.testing.assert_allclose(afqmc.local_energy(s, phi), e1, rtol=1e-12, atol=1e-12)


def test_thouless_theorem_convention():
    """exp(sum_ij A_ij E_ij)|phi> is the determinant exp(A) Phi (A complex, not symmetric)."""
    M, n_up, n_dn = 4, 2, 1
    E_up, E_dn = fci.one_body_operators(M, n_up, n_dn)
    rng = np.random.default_rng(1)
    A = 0.3 * (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M)))
    phi = random_phi(M, n_up + n_dn, 1, seed=4)[0]
    Ahat = np.einsum("ij,ijab->ab", A, E_up + E_dn)
    lhs = expm(Ahat) @ fci.determinant_vector(phi, n_up, n_dn)
    rhs = fci.determinant_vector(expm(A) @ phi, n_up, n_dn)
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)


def test_taylor_error_bound():
    rng = np.random.default_rng(2)
    M = 6
    A = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    A *= 0.2 / np.linalg.norm(A, 2)
    phi = random_phi(M, 3, 1, seed=8)[0]
    want = expm(A) @ phi
    for n in (2, 4, 6):
        got = afqmc.taylor_apply(A, phi, n)
        nrm = np.linalg.norm(A, 2)
        bound = nrm ** (n + 1) / np.math.factorial(n + 1) * np.exp(nrm) * np.linalg.norm(phi, 2) \
            if hasattr(np, "math") else None
        import math
        bound = nrm ** (n + 1) / math.factorial(n + 1) * math.exp(nrm) * np.linalg.norm(phi, 2)
        err = np.linalg.norm(got - want, 2)
        assert err <= bound
        assert err > 1e-3 * bound  # truncation really happens at order n


def _fci_split_propagator(s, n_up, n_dn):
    """exp(-dt H1/2) exp(-dt H2) exp(-dt H1/2) built in the many-body space from Eq. 1-3."""
    E_up, E_dn = fci.one_body_operators(s.M, n_up, n_dn)
    E = E_up + E_dn
    H = fci.hamiltonian(s.h1, s.L, n_up, n_dn)
    psi = fci.determinant_vector(s.trial, n_up, n_dn)
    D = H.shape[0]
    H2 = np.zeros((D, D), dtype=complex)
    for g in range(s.X):
        v = 1j * np.einsum("ik,ikab->ab", s.L[g], E)       # v_g of Sec. II.A
        vT = (psi @ v @ psi) / (psi @ psi)                  # <v_g> in the trial
        u = v - vT * np.eye(D)
        H2 += -0.5 * u @ u                                  # Eq. 2
    H1 = H - H2
    half = expm(-0.5 * s.dt * H1)
    return half @ expm(-s.dt * H2) @ half, psi


@pytest.mark.parametrize("shift", [0.0, 0.4 - 0.7j])
def test_hs_propagator_and_force_bias_by_quadrature(shift):
    """Gauss-Hermite average of one step equals exp(-dt H1/2) exp(-dt H2) exp(-dt H1/2).

    With a single Cholesky vector the Hubbard-Stratonovich integral (Eq. 4) is exact, so
    the quadrature must reproduce the split propagator of Eq. 3 in the many-body space.
    The force-bias shift with the factor exp(x xbar - xbar^2/2) (Eqs. 8-9, hybrid weight)
    leaves the integral unchanged for any constant complex xbar.
    """
    n_up, n_dn = 2, 1
    s = small_system(M=4, X=1, n_up=n_up, n_dn=n_dn, dt=0.05, mode=afqmc.FREE,
                     taylor_order=40, seed=31)
    P, psi = _fci_split_propagator(s, n_up, n_dn)
    phi = random_phi(s.M, s.N, 1, seed=12)
    phi /= np.abs(np.exp(afqmc.overlap(s, phi)[0])) ** (1 / s.N)
    t, wq = np.polynomial.hermite.hermgauss(80)
    xs = np.sqrt(2) * t
    wq = wq / np.sqrt(np.pi)
    n = xs.size
    phis = np.repeat(phi, n, axis=0)
    logO = afqmc.overlap(s, phis)
    xbar = np.full((n, 1), shift, dtype=complex)
    phi3, logO3, logR, logI = afqmc.step_determinant(s, phis, logO, xs[:, None], xbar)
    # walker weight w' = I (from w = 1): the represented state is w'|phi'>/<psi_T|phi'> * O(phi)
    acc = 0
    for q in range(n):
        vec = fci.determinant_vector(phi3[q], n_up, n_dn)
        acc = acc + wq[q] * np.exp(logI[q] - logO3[q] + logO[q]) * vec
    acc *= np.exp(-s.dt * s.E_T)
    want = P @ fci.determinant_vector(phi[0], n_up, n_dn)
    np.testing.assert_allclose(acc, want, rtol=0, atol=1e-11 * np.abs(want).max())


@pytest.mark.parametrize("n_up,n_dn", [(2, 2), (3, 1)])
def test_modified_gram_schmidt(n_up, n_dn):
    s = small_system(n_up=n_up, n_dn=n_dn)
    wk = afqmc.Walkers(s, 3, phi=random_phi(s.M, s.N, 3, seed=14))
    phi0 = wk.phi.copy()
    el0 = afqmc.local_energy(s, phi0)
    G0 = afqmc.green(s, phi0)
    logO0 = wk.logO.copy()
    afqmc.orthonormalise(s, wk)
    logr = np.zeros(3)
    for a, b in s.spins:
        Q = wk.phi[:, :, a:b]
        for k in range(3):
            np.testing.assert_allclose(Q[k].conj().T @ Q[k], np.eye(b - a), atol=1e-13)
            R = Q[k].conj().T @ phi0[k][:, a:b]
            np.testing.assert_allclose(np.tril(R, -1), 0, atol=1e-12)     # upper triangular
            assert np.all(np.abs(np.diag(R).imag) < 1e-12) and np.all(np.diag(R).real > 0)
            np.testing.assert_allclose(Q[k] @ R, phi0[k][:, a:b], atol=1e-12)
            logr[k] += np.sum(np.log(np.diag(R).real))
            # against LAPACK QR with the diagonal made positive
            q2, r2 = np.linalg.qr(phi0[k][:, a:b])
            ph = np.diag(r2) / np.abs(np.diag(r2))
            np.testing.assert_allclose(Q[k], q2 * ph[None, :], atol=1e-12)
    np.testing.assert_allclose(afqmc.local_energy(s, wk.phi), el0, rtol=1e-12)
    for Gs0, Gs1 in zip(G0, afqmc.green(s, wk.phi)):
        np.testing.assert_allclose(Gs1, Gs0, atol=1e-12)
    d = np.exp(wk.logO - (logO0 - logr))
    np.testing.assert_allclose(d, 1.0, atol=1e-12)


def test_non_interacting_limit_is_deterministic_closed_form():
    """L = 0: walkers follow exp(-tau h1) Psi exactly; weights and energies in closed form."""
    M, n_up, n_dn, dt = 6, 2, 1, 0.05
    h1, _ = make_hamiltonian(M, 1, 5)
    L = np.zeros((1, M, M))
    trial, _, _ = scf_trial(h1, L, n_up, n_dn)
    s = afqmc.System(h1, L, trial, n_up, n_dn, dt)
    wk = afqmc.Walkers(s, 2)
    lam, U = np.linalg.eigh(h1)
    rng = np.random.default_rng(0)
    for step in range(1, 21):
        afqmc.propagate(s, wk, rng.standard_normal((2, 1)))
        if step % 5 == 0:
            afqmc.orthonormalise(s, wk)
        tau = step * dt
        P = (U * np.exp(-tau * lam)) @ U.T
        w_want, e_want = np.exp(tau * s.E_T), 0.0
        for a, b in s.spins:
            Psi = trial[:, a:b]
            Ot = Psi.T @ P @ Psi
            w_want *= np.linalg.det(Ot)
            Th = P @ Psi @ np.linalg.inv(Ot)
            e_want += np.trace(Psi.T @ h1 @ Th)
        np.testing.assert_allclose(wk.w.real, w_want, rtol=1e-12)
        np.testing.assert_allclose(afqmc.local_energy(s, wk.phi).real, e_want, rtol=1e-12)
    assert abs(s.E_T - np.sum(np.linalg.eigvalsh(h1)[:2]) - lam[0]) < 1e-12


def test_walker_death_is_permanent_and_freezes_determinant():
    s = small_system(n_up=2, n_dn=1, scale=6.0, dt=0.05)
    wk = afqmc.Walkers(s, 64)
    rng = np.random.default_rng(3)
    dead_phi = {}
    for _ in range(30):
        afqmc.propagate(s, wk, rng.standard_normal((64, s.X)))
        for k in np.nonzero(~wk.alive)[0]:
            if k in dead_phi:
                np.testing.assert_array_equal(wk.phi[k], dead_phi[k])
            dead_phi[k] = wk.phi[k].copy()
            assert wk.w[k] == 0
    assert len(dead_phi) > 0


def test_force_bias_is_stationary_point_of_weight():
    """Eq. 8: with the optimal xbar the hybrid weight has no O(sqrt(dt)) dependence on x.

    d log I / d x_g at x = 0 is O(dt), while xbar itself is O(sqrt(dt)); a force bias of
    the wrong sign or scale leaves a derivative of order xbar.
    """
    s = small_system(n_up=2, n_dn=1, dt=1e-4, fb_cap=0.0)
    phi = random_phi(s.M, s.N, 1, seed=17)
    logO = afqmc.overlap(s, phi)
    xbar = afqmc.force_bias(s, afqmc.green(s, phi))
    eps = 1e-4
    for g in range(s.X):
        e = np.zeros((1, s.X))
        e[0, g] = eps
        lp = afqmc.step_determinant(s, phi, logO, e, xbar)[3][0]
        lm = afqmc.step_determinant(s, phi, logO, -e, xbar)[3][0]
        deriv = (lp - lm) / (2 * eps)
        assert abs(deriv) < 0.05 * abs(xbar[0, g]), (g, deriv, xbar[0, g])


def test_force_bias_cap():
    s = small_system(n_up=2, n_dn=1, dt=0.5, fb_cap=0.3)
    phi = random_phi(s.M, s.N, 4, seed=18)
    G = afqmc.green(s, phi)
    raw = -1j * s.sqrt_dt * (afqmc.rhobar(s, G) - s.rho_mf)
    xb = afqmc.force_bias(s, G)
    assert np.all(np.abs(xb) <= 0.3 + 1e-15)
    big = np.abs(raw) > 0.3
    assert np.any(big) and np.any(~big)
    np.testing.assert_allclose(xb[~big], raw[~big])
    np.testing.assert_allclose(xb[big] / np.abs(xb[big]), raw[big] / np.abs(raw[big]))
