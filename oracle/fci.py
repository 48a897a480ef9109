"""Brute-force many-body space for pinning the oracle (test infrastructure).

Determinant basis: per spin, occupation strings over M orbitals (bitmasks with
N_s bits), ordered by itertools.combinations.  A basis state is

    |S_up, S_dn> = prod_{i in S_up, ascending} c+_{i up} prod_{j in S_dn, ascending} c+_{j dn} |0>

with index iu * dim_dn + id.  The one-body excitation E^s_ij = c+_is c_js is built
on the strings with explicit fermionic signs; for spin down the up creators on
the left contribute (-1)^{N_up} twice, so E^dn = I_up (x) E_ij(string).

The Hamiltonian of Eq. 1 uses the anticommutation identity
    c+_is c+_jt c_lt c_ks = E^s_ik E^t_jl - delta_jk delta_st E^s_il,
checked term by term against a direct application of the four operators in
``two_body_direct``.
"""
import itertools
import numpy as np


def strings(M: int, n: int):
    return [sum(1 << i for i in occ) for occ in itertools.combinations(range(M), n)]


def _popcount_below(s: int, i: int) -> int:
    return bin(s & ((1 << i) - 1)).count("1")


def annihilate(s: int, j: int):
    """c_j |s> = sign |s'>; returns (sign, s') or (0, None)."""
    if not (s >> j) & 1:
        return 0, None
    return (-1) ** _popcount_below(s, j), s & ~(1 << j)


def create(s: int, i: int):
    if (s >> i) & 1:
        return 0, None
    return (-1) ** _popcount_below(s, i), s | (1 << i)


def string_one_body(M: int, n: int):
    """E[i, j] as dense [dim, dim] matrices on the n-electron strings of one spin."""
    S = strings(M, n)
    pos = {s: a for a, s in enumerate(S)}
    dim = len(S)
    E = np.zeros((M, M, dim, dim))
    for a, s in enumerate(S):
        for j in range(M):
            sj, s1 = annihilate(s, j)
            if sj == 0:
                continue
            for i in range(M):
                si, s2 = create(s1, i)
                if si == 0:
                    continue
                E[i, j, pos[s2], a] += sj * si
    return E


def one_body_operators(M: int, n_up: int, n_dn: int):
    """(E_up, E_dn): [M, M, D, D] spin-resolved excitation operators on the full space."""
    Eu = string_one_body(M, n_up)
    Ed = string_one_body(M, n_dn)
    du, dd = Eu.shape[2], Ed.shape[2]
    Iu, Id = np.eye(du), np.eye(dd)
    E_up = np.einsum("ijab,cd->ijacbd", Eu, Id).reshape(M, M, du * dd, du * dd)
    E_dn = np.einsum("ab,ijcd->ijacbd", Iu, Ed).reshape(M, M, du * dd, du * dd)
    return E_up, E_dn


def hamiltonian(h1, L, n_up: int, n_dn: int):
    """Dense H of Eq. 1 with V_ijkl = sum_g L^g_ik L^g_jl, in the determinant basis."""
    M = h1.shape[0]
    E_up, E_dn = one_body_operators(M, n_up, n_dn)
    E = E_up + E_dn
    H = np.einsum("ij,ijab->ab", h1, E)
    Q = np.einsum("gik,gkl->il", L, L)  # sum_k V_ikkl
    H -= 0.5 * np.einsum("il,ilab->ab", Q, E)
    for g in range(L.shape[0]):
        S = np.einsum("ik,ikab->ab", L[g], E)
        H += 0.5 * S @ S
    return H


def two_body_direct(V, M: int, n_up: int, n_dn: int):
    """1/2 sum V_ijkl sum_st c+_is c+_jt c_lt c_ks applied operator by operator (tiny M)."""
    Su, Sd = strings(M, n_up), strings(M, n_dn)
    # spin orbitals: up i -> i, down i -> M + i; state = up bits | (down bits << M)
    states = [u | (d << M) for u in Su for d in Sd]
    pos = {s: a for a, s in enumerate(states)}
    D = len(states)
    H = np.zeros((D, D))
    for a, s in enumerate(states):
        for i, j, k, l in itertools.product(range(M), repeat=4):
            v = V[i, j, k, l]
            if v == 0.0:
                continue
            for sg, tg in itertools.product((0, 1), repeat=2):
                sign = 1
                t = s
                for op, orb in (("a", k + sg * M), ("a", l + tg * M), ("c", j + tg * M),
                                ("c", i + sg * M)):
                    f = annihilate if op == "a" else create
                    sgn, t = f(t, orb)
                    if sgn == 0:
                        break
                    sign *= sgn
                else:
                    H[pos[t], a] += 0.5 * v * sign
    return H


def determinant_vector(phi, n_up: int, n_dn: int):
    """Coefficients det(Phi_up[S_up, :]) det(Phi_dn[S_dn, :]) of a determinant [M, N]."""
    M = phi.shape[0]
    cu = [np.linalg.det(phi[list(occ), :n_up]) if n_up else 1.0
          for occ in itertools.combinations(range(M), n_up)]
    cd = [np.linalg.det(phi[list(occ), n_up:]) if n_dn else 1.0
          for occ in itertools.combinations(range(M), n_dn)]
    return np.kron(np.array(cu), np.array(cd))


def ground_state(H):
    lam, U = np.linalg.eigh(H)
    return lam[0], U[:, 0]


def projected_energy(H, psi_T, taus):
    """E(tau) = <psi_T|H e^{-tau H}|psi_T> / <psi_T|e^{-tau H}|psi_T> (exact projection)."""
    lam, U = np.linalg.eigh(H)
    c = U.T @ psi_T
    out = []
    for tau in np.atleast_1d(taus):
        f = c * c * np.exp(-tau * (lam - lam[0]))
        out.append(np.sum(f * lam) / np.sum(f))
    return np.array(out)
