"""Real single-determinant trial from a plain SCF (input preparation).

The paper takes RHF/ROHF/UHF trials from NWChem (Sec. II.D).  Here the trial
for the synthetic Hamiltonian comes from a Roothaan iteration with Pulay DIIS,
started from the eigenvectors of h1:

  F^s = h1 + J - K^s,  J = sum_g L_g tr(L_g P),  K^s = sum_g (L_g C_s)(L_g C_s)^T
  P = P^up + P^dn,  P^s = C_s C_s^T  (C_s: the N_s lowest orbitals of F^s)

RHF (one shared orbital set) when N_up == N_dn, UHF otherwise.  When the plain
iteration does not settle within ``max_iter`` steps (a small gap between the
highest occupied and lowest virtual orbitals makes DIIS oscillate, as for the
M = 200 shapes whose one-body levels are 0.025 Ha apart), it restarts from the
h1 eigenvectors with the virtual orbitals shifted up by ``level_shift`` Ha
(F + b (I - P) is diagonalised; the converged orbitals are those of F) for up to
``shift_iter`` steps.  If neither settles, the lowest-energy determinant visited
is returned (deterministic for a given Hamiltonian).  The trial is the
M x (N_up + N_dn) matrix [Psi_up | Psi_dn] with orthonormal columns.
"""
import numpy as np


def _fock(h1, L, C_up, C_dn):
    X, M, _ = L.shape
    Lf = L.reshape(X, M * M)
    P = C_up @ C_up.T + C_dn @ C_dn.T
    J = (Lf.T @ (Lf @ P.T.reshape(M * M))).reshape(M, M)      # sum_g L_g tr(L_g P)
    out = []
    for C in (C_up, C_dn):
        ns = C.shape[1]
        if ns == 0:
            out.append(h1 + J)
            continue
        LC = (L.reshape(X * M, M) @ C).reshape(X, M, ns)        # L_g C
        W = LC.transpose(1, 0, 2).reshape(M, X * ns)
        out.append(h1 + J - W @ W.T)                            # sum_g (L_g C)(L_g C)^T
    return out


def _energy(h1, F, C_up, C_dn):
    e = 0.0
    for C, Fs in zip((C_up, C_dn), F):
        e += 0.5 * np.sum((h1 + Fs) * (C @ C.T))
    return float(e)


def hf_energy(h1, L, C_up, C_dn):
    return _energy(h1, _fock(h1, L, C_up, C_dn), C_up, C_dn)


def _roothaan(h1, L, n_up, n_dn, max_iter, tol, n_diis, shift):
    """DIIS Roothaan iteration from the h1 eigenvectors, virtual orbitals shifted by ``shift``.
    Returns (best energy, orbitals [C_up, C_dn], converged, iterations)."""
    M = h1.shape[0]
    restricted = n_up == n_dn

    def occ(F, n):
        _, V = np.linalg.eigh(F)
        return V[:, :n].copy()

    _, V = np.linalg.eigh(h1)
    C = [V[:, :n_up].copy(), V[:, :n_dn].copy()]
    best = (np.inf, C)
    hist_F, hist_e = [], []
    it = 0
    for it in range(1, max_iter + 1):
        F = _fock(h1, L, C[0], C[1])
        e = _energy(h1, F, C[0], C[1])
        if restricted:
            Fa = 0.5 * (F[0] + F[1])
            F = [Fa, Fa]
        if e < best[0]:
            best = (e, [C[0].copy(), C[1].copy()])
        P = [C[0] @ C[0].T, C[1] @ C[1].T]
        err = np.concatenate([(F[s] @ P[s] - P[s] @ F[s]).ravel() for s in range(2)])
        if np.max(np.abs(err)) < tol:
            return e, C, True, it
        hist_F.append([F[0].copy(), F[1].copy()])
        hist_e.append(err)
        hist_F, hist_e = hist_F[-n_diis:], hist_e[-n_diis:]
        n = len(hist_F)
        if n >= 2:
            B = -np.ones((n + 1, n + 1))
            B[n, n] = 0.0
            E = np.array(hist_e)
            B[:n, :n] = E @ E.T
            rhs = np.zeros(n + 1)
            rhs[n] = -1.0
            try:
                coef = np.linalg.solve(B, rhs)[:n]
                F = [sum(c * f[s] for c, f in zip(coef, hist_F)) for s in range(2)]
            except np.linalg.LinAlgError:
                pass
        if shift:
            F = [F[s] + shift * (np.eye(M) - P[s]) for s in range(2)]
        C = [occ(F[0], n_up), occ(F[1], n_dn)]
    return best[0], best[1], False, it


def scf_trial(h1, L, n_up: int, n_dn: int, max_iter: int = 60, tol: float = 1e-10,
              n_diis: int = 8, level_shift: float = 0.1, shift_iter: int = 400):
    """Return (trial [M, n_up+n_dn], converged: bool, n_iter: int)."""
    M = h1.shape[0]
    if not (0 <= n_dn <= M and 0 <= n_up <= M):
        raise ValueError("occupations out of range")
    e, C, converged, it = _roothaan(h1, L, n_up, n_dn, max_iter, tol, n_diis, 0.0)
    if not converged and level_shift > 0 and shift_iter > 0:
        e2, C2, converged, it2 = _roothaan(h1, L, n_up, n_dn, shift_iter, tol, n_diis, level_shift)
        it += it2
        if converged or e2 < e:
            C = C2
    if n_up == n_dn:
        C = [C[0], C[0].copy()]
    trial = np.concatenate(C, axis=1)
    # sign convention: each orbital's largest-magnitude coefficient positive (ties: the first).
    # Nothing of one system depends on its orbitals' signs; the overlap ratio between two
    # systems' trials that seeds a secondary system does (its sign is that of the product of
    # the flips), and a common convention makes it that of the physical overlap.
    for j in range(trial.shape[1]):
        k = int(np.argmax(np.abs(trial[:, j])))
        if trial[k, j] < 0:
            trial[:, j] = -trial[:, j]
    return np.ascontiguousarray(trial), converged, it
