"""Checkpoints of a walker population for resuming a run.

Between steps the state of a system is its walkers Phi, their weights w and the step
counter t. The fields x_{t,k,g} are a function of (seed, t, pair index k, g) alone, so a
handle with the same Hamiltonian, seed and walker offset that is given (Phi, w, t) back draws
exactly the fields the interrupted run would have drawn. log O and Theta are recomputed from
Phi on restore. A checkpoint taken right after an orthonormalisation therefore resumes an
FP64 run bit for bit; see afqmc_set_step in include/afqmc.h.

Files are plain ``.npz`` archives, written and read without pickling.
"""
import numpy as np

# identity of the run a checkpoint belongs to: (M, X, n_up, n_dn, n_walkers, n_repeats,
# seed, walker_offset, precision, mode)
_KEYS = ("M", "X", "n_up", "n_dn", "n_walkers", "n_repeats", "seed", "walker_offset",
         "precision", "mode")


def identity(system):
    """The identity tuple of a System (or any object with the same attributes)."""
    o = system.opt
    return np.array([system.M, system.X, system.n_up, system.n_dn, system.n_walkers,
                     system.n_repeats, o.seed, o.walker_offset, o.precision, o.mode],
                    dtype=np.uint64)


def make(system, phi, w, step):
    """Checkpoint dict for ``system`` from its walkers phi [Nw, M, N] (complex), weights w
    [Nw] (complex) and step counter."""
    phi = np.asarray(phi, dtype=np.complex128)
    w = np.asarray(w, dtype=np.complex128)
    ident = identity(system)
    nw, M, N = int(ident[4]), int(ident[0]), int(ident[2] + ident[3])
    if phi.shape != (nw, M, N) or w.shape != (nw,):
        raise ValueError(f"checkpoint shapes {phi.shape}, {w.shape} do not match "
                         f"({nw}, {M}, {N}) walkers")
    if step < 0:
        raise ValueError("step must be >= 0")
    return dict(identity=ident, phi=phi, w=w, step=np.uint64(step))


def check(ck, system):
    """Raise ValueError unless checkpoint ``ck`` belongs to a run like ``system``'s."""
    got, want = np.asarray(ck["identity"], dtype=np.uint64), identity(system)
    if got.shape != want.shape or not np.array_equal(got, want):
        diff = [k for k, a, b in zip(_KEYS, got, want) if a != b] if got.shape == want.shape \
            else ["layout"]
        raise ValueError(f"checkpoint does not match this system (differs in {', '.join(diff)})")


def save(path, ck):
    """Write checkpoint ``ck`` to ``path`` (.npz)."""
    np.savez(path, identity=ck["identity"], phi=ck["phi"], w=ck["w"],
             step=np.asarray(ck["step"], dtype=np.uint64))


def load(path):
    """Read a checkpoint written by save()."""
    with np.load(path, allow_pickle=False) as z:
        return dict(identity=z["identity"], phi=z["phi"], w=z["w"], step=np.uint64(z["step"]))
