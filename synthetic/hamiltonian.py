"""Synthetic molecular-like Hamiltonian in an orthonormal basis of M orbitals.

Recipe (stated once, used by every test and by the benchmark):

* h1 = diag(linspace(-2, 3, M)) plus a symmetric off-diagonal part with
  entries N(0, (0.05 exp(-|i-j|/4))^2), drawn for i < j and mirrored.
* X Cholesky vectors L_g (g = 0..X-1), each symmetric M x M with entries
  N(0, (0.3 exp(-4 g / X))^2), drawn for i <= j and mirrored.
  The two-body matrix elements are then V_ijkl = sum_g L^g_ik L^g_jl (Sec. II.A).
* Generator: numpy PCG64 seeded with ``seed`` (default 1703); draws are made in
  the order h1 off-diagonal block first, then L_0 .. L_{X-1}, each as a full
  M x M standard-normal block of which the upper triangle is kept.
* Nuclear repulsion is zero.
* ``coupling`` multiplies every L_g (default 1: the recipe as stated).  With the
  recipe as stated, sum_g Var(L^g_ij) = 0.09 sum_g exp(-8g/X) grows like X, and
  for X >= 320 the one-body exponent sqrt(dt) sum_g x_g L_g of a step has norm of
  order 2, so that every phaseless walker dies within ~10 steps.
  ``moderate_coupling(X) = sqrt(6 / X)`` keeps that variance at ~0.07 Ha for any
  X; runs that need long-lived walkers (long-run statistics) use it.  The arithmetic
  per step does not depend on the values, so throughput is the same either way.
"""
import numpy as np


def moderate_coupling(X: int) -> float:
    return float(np.sqrt(6.0 / max(X, 1)))


def make_hamiltonian(M: int, X: int, seed: int = 1703, coupling: float = 1.0):
    """Return (h1 [M,M], L [X,M,M]) as float64 arrays."""
    if M < 1 or X < 0:
        raise ValueError("M >= 1 and X >= 0 required")
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = np.arange(M)
    sd = 0.05 * np.exp(-np.abs(idx[:, None] - idx[None, :]) / 4.0)
    off = np.triu(rng.standard_normal((M, M)) * sd, 1)
    h1 = np.diag(np.linspace(-2.0, 3.0, M)) + off + off.T
    L = np.empty((X, M, M))
    scale = 0.3 * np.exp(-4.0 * np.arange(X) / max(X, 1))
    for g in range(X):
        u = np.triu(rng.standard_normal((M, M)) * scale[g])
        L[g] = u + np.triu(u, 1).T
    if coupling != 1.0:
        L *= coupling
    return h1, L
