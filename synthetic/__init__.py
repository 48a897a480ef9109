"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package holds none of the AFQMC method's arithmetic.  It produces the inputs
the method consumes:

* ``hamiltonian``: the model one-body matrix h1 and symmetric Cholesky vectors
  L_g of the Hamiltonian of Eq. 1 (the paper's molecules and their NWChem
  Cholesky vectors are not available; this generator stands in for them with
  the paper's shape relations, Nchol of order 5-10 M).
* ``scf``: a plain Roothaan (RHF/UHF) iteration giving the real single-
  determinant trial, playing the role of the paper's HF trial (Sec. II.D).
* ``fields``: seeded standard-normal auxiliary-field blocks for parity runs
  that pass explicit fields to both sides.
* ``configs``: the five synthetic workload shapes.
"""
from .hamiltonian import make_hamiltonian
from .scf import scf_trial
from .fields import explicit_fields
from .configs import CONFIGS, build_system

__all__ = ["make_hamiltonian", "scf_trial", "explicit_fields", "CONFIGS", "build_system"]
