"""Preliminary equilibration scheme (PES, Sec. II.C) and the population control it uses.

TEST INFRASTRUCTURE ONLY, like the rest of the oracle package: plain FP64 NumPy that shares
no code with the CUDA path.

PES. The primary system A is first equilibrated on its own, with population control. The
secondary system B then starts from A's determinants. Each weight is multiplied by the ratio
of the two trial overlaps <psi_T^B|phi> / <psi_T^A|phi>, and the ratio's phase is projected
out. Both systems then run on correlated fields without population control, and the energy
difference is measured.

Readings (the paper names the steps, not their details):
* Population control is the comb. Within each repeat, the n walkers of total weight W are
  replaced by the n walkers found at the points (j + u) W / n, j = 0 .. n-1, of the running
  sum of the weights (summed left to right, W its last value), with one uniform u per
  repeat. Every copy carries weight W / n. A dead walker (w = 0) is never chosen. The paper
  says only that walkers of large weight are replicated and walkers of small weight removed.
* "Phases projected" is the phaseless projection of the ratio R: w_B = w_A |R| max(0, cos arg R).
* When B has fewer electrons of a spin (an ion seeded from the neutral), its walker keeps the
  first N_s^B columns of that spin block. These are the propagated images of the trial's
  first orbitals, so the electron is removed from the last occupied trial orbital. A
  secondary system with more electrons than the primary is not supported.
"""
import numpy as np

from . import afqmc
from .philox import gaussian_fields


def comb_select(w, n_out, u):
    """Comb over weights w (>= 0): indices of the n_out walkers found at the points
    (j + u) W / n_out, j = 0 .. n_out - 1, of the running sum, and the common new weight."""
    w = np.asarray(w, dtype=np.float64)
    if np.any(w < 0):
        raise ValueError("comb weights must be >= 0")
    cum = np.cumsum(w)                 # left to right; W is its last value, so the total and
    W = float(cum[-1]) if w.size else 0.0   # the running sums share one rounding order
    if not W > 0:
        raise ValueError("no weight to comb")
    points = (np.arange(n_out) + float(u)) * (W / n_out)
    # first walker whose running sum exceeds the point: zero weights are stepped over
    idx = np.searchsorted(cum, points, side="right")
    return np.minimum(idx, w.size - 1), W / n_out


def population_control(sys: afqmc.System, wk: afqmc.Walkers, groups, n_repeats, u):
    """Comb each repeat's walkers in place (phaseless weights); u [n_repeats] in [0, 1)."""
    if sys.mode != afqmc.PHASELESS:
        raise ValueError("population control is defined here for real (phaseless) weights")
    for r in range(n_repeats):
        m = np.nonzero(np.asarray(groups) == r)[0]
        if m.size == 0:
            continue
        w = np.where(wk.alive[m], wk.w[m].real, 0.0)
        pick, w_new = comb_select(w, m.size, u[r])
        src = m[pick]
        wk.phi[m] = wk.phi[src]
        wk.logO[m] = wk.logO[src]
        wk.w[m] = w_new
        wk.alive[m] = True


def seed_columns(sysA: afqmc.System, sysB: afqmc.System):
    """Columns of A's walkers that form B's walker (spin-up block first, then spin-down)."""
    if sysB.M != sysA.M or sysB.n_up > sysA.n_up or sysB.n_dn > sysA.n_dn:
        raise ValueError("the secondary system needs the same basis and no more electrons "
                         "of either spin than the primary")
    return list(range(sysB.n_up)) + list(range(sysA.n_up, sysA.n_up + sysB.n_dn))


def seed_secondary(sysA: afqmc.System, sysB: afqmc.System, wkA: afqmc.Walkers):
    """B's walkers from A's: the determinants (columns per seed_columns) and the weights
    w_B = w_A |R| max(0, cos arg R), R = <psi_T^B|phi_B> / <psi_T^A|phi_A>."""
    phi = wkA.phi[:, :, seed_columns(sysA, sysB)]
    logR = afqmc.overlap(sysB, phi) - wkA.logO
    w = wkA.w.real * np.exp(logR.real) * np.maximum(0.0, np.cos(logR.imag))
    w = np.where(wkA.alive, w, 0.0)
    return afqmc.Walkers(sysB, phi.shape[0], phi=phi, w=w.astype(np.complex128))


def run_pes(sysA: afqmc.System, sysB: afqmc.System, n_walkers: int, n_eq: int, n_steps: int,
            seed: int, u, pc_every: int = 5, energy_every: int = 5, mgs_every: int = 5,
            n_repeats: int = 1):
    """The whole scheme. A runs n_eq steps alone (fields of steps 0 .. n_eq - 1), with its
    population combed after every pc_every steps using u [n_eq // pc_every, n_repeats]. B is
    seeded from A, and both run n_steps more on the shared fields of steps n_eq, n_eq + 1, ...
    without population control. Returns run_pair's dict for the correlated part."""
    k = np.arange(n_walkers)
    groups = afqmc.repeat_groups(n_walkers, n_repeats)
    wkA = afqmc.Walkers(sysA, n_walkers)
    n_pc = 0
    for t in range(n_eq):
        afqmc.propagate(sysA, wkA, gaussian_fields(seed, t, k, sysA.X))
        if mgs_every and (t + 1) % mgs_every == 0:
            afqmc.orthonormalise(sysA, wkA)
        if pc_every and (t + 1) % pc_every == 0:
            population_control(sysA, wkA, groups, n_repeats, u[n_pc])
            n_pc += 1
    wkB = seed_secondary(sysA, sysB, wkA)
    return afqmc.run_pair(sysA, sysB, n_walkers, n_steps, seed, energy_every=energy_every,
                          mgs_every=mgs_every, n_repeats=n_repeats, walkers=(wkA, wkB),
                          t0=n_eq)
