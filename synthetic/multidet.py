"""Multi-determinant trial for the synthetic Hamiltonian (input preparation).

The paper's multi-determinant trials are CASSCF expansions from PySCF, truncated by the size
of their CI coefficients (Sec. II.D; the tables of Sec. III).  This stands in for them:

* orbitals: the canonical orbitals of the SCF trial, one orthonormal set C (the eigenvectors of
  the spin-averaged Fock matrix of the converged SCF determinant);
* CI: the exact ground state of H (Eq. 1) among all determinants built from the lowest
  ``n_orb`` of those orbitals (a CASCI with every electron active; the Hamiltonian in that
  orbital subset is h1 and L rotated by C and truncated);
* truncation: the determinants whose coefficient has magnitude >= ``threshold`` (at most
  ``max_det`` of them, largest first), as in the paper's minimum-CI-coefficient cut;
* walkers start from the determinant of the lowest eigenvectors of h1 (the core-Hamiltonian
  guess), which overlaps every determinant of the expansion; a walker sitting on a determinant
  of the orthonormal expansion would be orthogonal to all the others.

Determinant d is the real M x N matrix [C[:, S_up] | C[:, S_dn]] of its occupied orbitals
(ascending), i.e. the many-body basis state prod_{i in S_up} c+_i,up prod_{j in S_dn} c+_j,dn |0>
of the rotated orbitals, with its CI coefficient.  None of the method's arithmetic is here.
"""
import itertools

import numpy as np

from .scf import _fock


def _spin_strings(n_orb, n):
    """Occupation tuples (ascending) of n electrons in n_orb orbitals, in combinations order."""
    return list(itertools.combinations(range(n_orb), n))


def _hop(occ, i, j):
    """c+_i c_j applied to the ordered occupation tuple occ: (sign, new tuple) or (0, None).
    The sign counts the occupied orbitals the operators pass on their way to their slots."""
    if j not in occ:
        return 0, None
    rest = [o for o in occ if o != j]
    sign = (-1) ** occ.index(j)
    if i in rest:
        return 0, None
    pos = sum(1 for o in rest if o < i)
    return sign * (-1) ** pos, tuple(sorted(rest + [i]))


def _excitations(n_orb, n):
    """E[i][j]: dense [ns, ns] matrix of c+_i c_j on the strings of one spin."""
    S = _spin_strings(n_orb, n)
    idx = {s: a for a, s in enumerate(S)}
    E = np.zeros((n_orb, n_orb, len(S), len(S)))
    for a, s in enumerate(S):
        for i in range(n_orb):
            for j in range(n_orb):
                sg, t = _hop(s, i, j)
                if sg:
                    E[i, j, idx[t], a] = sg
    return E


def _cas_hamiltonian(h1, L, n_up, n_dn):
    """H of Eq. 1 on the determinants of a small orbital set (basis |S_up> x |S_dn>, up
    creators first): sum_ij h_ij E_ij + 1/2 sum_ijkl V_ijkl c+_i c+_j c_l c_k with
    V_ijkl = sum_g L_g,ik L_g,jl, written as 1/2 sum_g (sum_ik L_g,ik E_ik)^2 minus the
    one-body term 1/2 sum_ik (sum_g L_g L_g)_ik E_ik that normal ordering leaves."""
    n_orb = h1.shape[0]
    Eu, Ed = _excitations(n_orb, n_up), _excitations(n_orb, n_dn)
    du, dd = Eu.shape[2], Ed.shape[2]
    # spin-summed E_ij on the product basis (down strings fastest; the down operators pass
    # an even number of up creators twice, so they carry no extra sign)
    E = np.einsum("ijab,cd->ijacbd", Eu, np.eye(dd)) + np.einsum("ab,ijcd->ijacbd", np.eye(du), Ed)
    E = E.reshape(n_orb, n_orb, du * dd, du * dd)
    H = np.einsum("ij,ijab->ab", h1 - 0.5 * np.einsum("gik,gkj->ij", L, L), E)
    for g in range(L.shape[0]):
        Sg = np.einsum("ik,ikab->ab", L[g], E)
        H += 0.5 * Sg @ Sg
    return H


def canonical_orbitals(h1, L, trial, n_up, n_dn):
    """Eigenvectors (ascending) of the spin-averaged Fock matrix of the determinant `trial`."""
    F = _fock(h1, L, trial[:, :n_up], trial[:, n_up:])
    _, C = np.linalg.eigh(0.5 * (F[0] + F[1]))
    return C


def cas_trial(h1, L, trial, n_up, n_dn, n_orb, threshold=0.01, max_det=64):
    """(dets [Nd, M, N], coeffs [Nd], start [M, N], info) of a truncated CASCI trial."""
    M = h1.shape[0]
    if not (max(n_up, n_dn) <= n_orb <= M):
        raise ValueError("n_orb must hold every electron and fit the basis")
    C = canonical_orbitals(h1, L, trial, n_up, n_dn)
    Cs = C[:, :n_orb]
    hs = Cs.T @ h1 @ Cs
    Ls = np.einsum("ia,gij,jb->gab", Cs, L, Cs)
    H = _cas_hamiltonian(hs, Ls, n_up, n_dn)
    lam, U = np.linalg.eigh(H)
    ci = U[:, 0]
    ups = list(itertools.combinations(range(n_orb), n_up))
    dns = list(itertools.combinations(range(n_orb), n_dn))
    order = np.argsort(-np.abs(ci), kind="stable")
    keep = [k for k in order if abs(ci[k]) >= threshold][:max_det]
    if not keep:
        keep = [int(order[0])]
    dets, coeffs = [], []
    for k in keep:
        su, sd = ups[k // len(dns)], dns[k % len(dns)]
        dets.append(np.concatenate([Cs[:, list(su)], Cs[:, list(sd)]], axis=1))
        coeffs.append(ci[k])
    coeffs = np.array(coeffs)
    coeffs /= np.linalg.norm(coeffs)
    V = np.linalg.eigh(h1)[1]
    start = np.concatenate([V[:, :n_up], V[:, :n_dn]], axis=1)
    info = dict(e_casci=float(lam[0]), n_space=int(H.shape[0]), weight=float(
        np.sum(ci[keep] ** 2)))
    return np.ascontiguousarray(np.array(dets)), coeffs, np.ascontiguousarray(start), info
