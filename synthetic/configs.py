"""The five synthetic workload shapes (pairs share one field stream).

C1  M=8,   X=24,   2/2 vs 2/1,  128 walkers x 400 steps, dt=0.01   (FCI-checkable)
C2  M=64,  X=320,  8/8 vs 8/7,  2048 walkers x 2000 steps, dt=0.005 (FP64 throughput)
C3  M=128, X=768,  16/16 vs 16/15, 4096 walkers                       (mixed + batched)
C4  A: M=200, X=1000, 9/9; B: M=190, X=950, 8/8 (B drawn with seed+1000), 2048 walkers,
    1000 steps, dt=0.005 (uneven pair)
C5  M=96,  X=480,  12/12, 1024 walkers x 200 steps (adjoint)
Energy measurement and modified Gram-Schmidt every 5 steps in all of them.
"""
from .hamiltonian import make_hamiltonian, moderate_coupling
from .scf import scf_trial

CONFIGS = {
    "C1": dict(A=dict(M=8, X=24, n_up=2, n_dn=2, seed=1703),
               B=dict(M=8, X=24, n_up=2, n_dn=1, seed=1703),
               n_walkers=128, n_steps=400, dt=0.01),
    "C2": dict(A=dict(M=64, X=320, n_up=8, n_dn=8, seed=1703),
               B=dict(M=64, X=320, n_up=8, n_dn=7, seed=1703),
               n_walkers=2048, n_steps=2000, dt=0.005),
    "C3": dict(A=dict(M=128, X=768, n_up=16, n_dn=16, seed=1703),
               B=dict(M=128, X=768, n_up=16, n_dn=15, seed=1703),
               n_walkers=4096, n_steps=1000, dt=0.005),
    "C4": dict(A=dict(M=200, X=1000, n_up=9, n_dn=9, seed=1703),
               B=dict(M=190, X=950, n_up=8, n_dn=8, seed=2703),
               n_walkers=2048, n_steps=1000, dt=0.005),
    "C5": dict(A=dict(M=96, X=480, n_up=12, n_dn=12, seed=1703),
               B=None, n_walkers=1024, n_steps=200, dt=0.005),
}

_cache = {}


def build_system(M, X, n_up, n_dn, seed=1703, coupling=1.0):
    """Return dict(h1, L, trial, n_up, n_dn, M, X) for one system (cached).

    ``coupling``: 1.0 is the recipe as stated; the string "moderate" selects
    ``moderate_coupling(M, X)`` (long-lived walkers for long-run statistics).
    """
    if coupling == "moderate":
        coupling = moderate_coupling(M, X)
    key = (M, X, n_up, n_dn, seed, float(coupling))
    if key not in _cache:
        h1, L = make_hamiltonian(M, X, seed, coupling=coupling)
        trial, ok, _ = scf_trial(h1, L, n_up, n_dn)
        _cache[key] = dict(h1=h1, L=L, trial=trial, n_up=n_up, n_dn=n_dn, M=M, X=X,
                           scf_converged=ok, coupling=float(coupling))
    return _cache[key]
