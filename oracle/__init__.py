"""Plain FP64 CPU oracle for correlated-sampling phaseless AFQMC.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only the tests, the smoke check of ``__graft_entry__``
and the CPU-baseline leg of ``bench.py`` use it.  It shares no code with the
CUDA path; the two meet only in the seeded inputs of the ``synthetic``
package.

Modules
  philox  -- Philox-4x32-10 counter-based generator and Box-Muller normals
             (from the published definitions; Salmon et al., SC'11; Box and
             Muller 1958).
  afqmc   -- the walker propagation of Sec. II.A-B (Eqs. 1-11), one step at a
             time, in the paper's order and notation, complex128/float64.
  fci     -- brute-force many-body space (determinant strings) used to pin the
             oracle: dense H of Eq. 1, FCI energies, determinant expansions.
  stats   -- repeat statistics of Sec. II.B (mean/SE among repeats,
             cumulative averages after equilibration, earliest minimum SE)
             and the Flyvbjerg-Petersen reblocking error estimate.

Parity status: every function is pinned by a ``-m "not gpu"`` test against a
closed form, an invariant, brute force in the many-body space or published
known-answer vectors, except the phaseless-bias size of the energy itself,
which has no closed form ("parity unpinned" for the phaseless energy value
against FCI: reported, not asserted).
"""
