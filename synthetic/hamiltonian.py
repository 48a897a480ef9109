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
  recipe as stated, the one-body matrix of a step's fields, sum_g x_g L_g (x_g ~ N(0, 1)),
  has entries of variance sigma_1^2 = 0.09 sum_g exp(-8 g / X), which grows like X, and a
  spectral norm near 2 sigma_1 sqrt(M) (the semicircle edge of a symmetric random matrix).
  At X >= 320 the exponent sqrt(dt) sum_g x_g L_g of a step then has norm of order 2, the
  order-6 Taylor series is inaccurate and every phaseless walker dies within ~10 steps.
  ``moderate_coupling(M, X)`` scales L so that the expected spectral norm of
  sum_g x_g L_g is STEP_NORM = 2 sqrt(2) for every shape: sqrt(dt) times it is 0.2 at the
  time step dt = 0.005 of every workload that uses it.  The norm measures how far one step
  rotates a walker, and walkers that drift faster lose their phase sooner: held fixed
  across the shapes, more than 90% of the walkers of the M = 64..200 pairs live to
  tau = 2.  The arithmetic per step does not depend on the values, so throughput is the
  same either way.
"""
import numpy as np


STEP_NORM = 2.0 * np.sqrt(2.0)


def field_entry_sd(X: int) -> float:
    """Standard deviation of an entry of sum_g x_g L_g at coupling 1 (x_g ~ N(0, 1))."""
    return float(np.sqrt(0.09 * np.sum(np.exp(-8.0 * np.arange(X) / max(X, 1)))))


def moderate_coupling(M: int, X: int) -> float:
    """Scale of every L_g that puts the expected spectral norm of sum_g x_g L_g at
    STEP_NORM, from its semicircle estimate 2 sigma_1 sqrt(M)."""
    return float(STEP_NORM / (2.0 * np.sqrt(M) * field_entry_sd(X)))


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
