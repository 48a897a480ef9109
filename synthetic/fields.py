"""Explicit auxiliary-field blocks for parity runs.

Parity tests can hand both the oracle and the CUDA path the same pre-drawn
standard-normal fields x[t, k, g] instead of the counter-based stream.  These
come from numpy PCG64 and involve none of the method's arithmetic.
"""
import numpy as np


def explicit_fields(n_steps: int, n_walkers: int, X: int, seed: int = 7):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((n_steps, n_walkers, X))
