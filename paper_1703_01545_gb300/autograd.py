"""torch.autograd wrappers of the library's derivatives of a run's mixed energy.

``mixed_energy(lam, ...)`` runs the FP64 propagation of one system with h1 + lam P on a
fixed field realisation and returns the run's mixed energy (the mean of the per-measurement
estimates of Eq. 7); its backward pass uses dE/dlambda from the library's tangent mode, so
torch.autograd.grad gives the exact derivative of that estimate along P.

``mixed_energy_h1(h1, ...)`` returns the same estimate as a function of the whole h1 tensor;
its backward pass is the library's checkpointed reverse mode (one forward run, one reverse
sweep), giving dE/dh1 for all M^2 entries at once.
"""
import numpy as np
import torch

from .api import FP64, System


class _MixedEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, lam, h1, L, trial, n_up, n_dn, P, fields, dt, n_walkers, n_steps,
                mgs_every, energy_every, seed):
        lv = float(lam.detach().cpu())
        s = System(h1 + lv * P, L, trial, n_up, n_dn, dt=dt, n_walkers=n_walkers, seed=seed,
                   precision=FP64)
        s.set_tangent(P)
        es, ds = [], []
        for t in range(n_steps):
            s.propagate(1, None if fields is None else fields[t:t + 1])
            if mgs_every and (t + 1) % mgs_every == 0:
                s.orthonormalise()
            if energy_every and (t + 1) % energy_every == 0:
                em, dm, _ = s.energy_tangent()
                es.append(em[0])
                ds.append(dm[0])
        s.close()
        ctx.dE = float(np.mean(ds))
        return torch.tensor(float(np.mean(es)), dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad):
        return (grad * ctx.dE,) + (None,) * 13


def mixed_energy(lam, h1, L, trial, n_up, n_dn, P, fields=None, dt=0.01, n_walkers=128,
                 n_steps=20, mgs_every=5, energy_every=5, seed=1):
    """Mixed energy of a run with h1 + lam P (differentiable in the scalar tensor lam)."""
    return _MixedEnergy.apply(lam, np.asarray(h1, float), np.asarray(L, float),
                              np.asarray(trial, float), int(n_up), int(n_dn), np.asarray(P, float),
                              None if fields is None else np.ascontiguousarray(fields, float),
                              float(dt), int(n_walkers), int(n_steps), int(mgs_every),
                              int(energy_every), int(seed))


def mixed_energy_grad_h1(h1, L, trial, n_up, n_dn, fields=None, dt=0.01, n_walkers=128,
                         n_steps=20, mgs_every=5, energy_every=5, seed=1):
    """dE/dh1 [M][M] (symmetric) of the same estimate, one tangent run per symmetric basis
    direction (E_ij + E_ji for i < j, E_ii on the diagonal): M(M+1)/2 forward runs."""
    h1 = np.asarray(h1, float)
    M = h1.shape[0]
    grad = np.zeros((M, M))
    for i in range(M):
        for j in range(i, M):
            P = np.zeros((M, M))
            P[i, j] = P[j, i] = 1.0
            s = System(h1, L, trial, n_up, n_dn, dt=dt, n_walkers=n_walkers, seed=seed,
                       precision=FP64)
            s.set_tangent(P)
            ds = []
            for t in range(n_steps):
                s.propagate(1, None if fields is None else fields[t:t + 1])
                if mgs_every and (t + 1) % mgs_every == 0:
                    s.orthonormalise()
                if energy_every and (t + 1) % energy_every == 0:
                    ds.append(s.energy_tangent()[1][0])
            s.close()
            g = float(np.mean(ds))
            if i == j:
                grad[i, i] = g
            else:   # direction E_ij + E_ji: split equally over the symmetric pair
                grad[i, j] = grad[j, i] = 0.5 * g
    return grad


class _MixedEnergyH1(torch.autograd.Function):
    @staticmethod
    def forward(ctx, h1, L, trial, n_up, n_dn, fields, dt, n_walkers, n_steps, mgs_every,
                energy_every, seed, checkpoint):
        hv = h1.detach().to("cpu", torch.float64).numpy()
        s = System(hv, L, trial, n_up, n_dn, dt=dt, n_walkers=n_walkers, seed=seed,
                   precision=FP64)
        try:
            E, G = s.adjoint_run(n_steps, fields, mgs_every=mgs_every, energy_every=energy_every,
                                 checkpoint=checkpoint)
        finally:
            s.close()
        ctx.save_for_backward(torch.from_numpy(G).to(device=h1.device, dtype=h1.dtype))
        return torch.tensor(E, dtype=h1.dtype, device=h1.device)

    @staticmethod
    def backward(ctx, grad):
        (G,) = ctx.saved_tensors
        return (grad * G,) + (None,) * 12


def mixed_energy_h1(h1, L, trial, n_up, n_dn, fields=None, dt=0.01, n_walkers=128, n_steps=20,
                    mgs_every=5, energy_every=5, seed=1, checkpoint=0):
    """Mixed energy of a run as a differentiable function of the h1 tensor [M, M] (float64).
    The gradient treats the M^2 entries as independent; checkpoint=0 picks about
    sqrt(n_steps) steps per recomputed segment."""
    return _MixedEnergyH1.apply(h1, np.asarray(L, float), np.asarray(trial, float), int(n_up),
                                int(n_dn),
                                None if fields is None else np.ascontiguousarray(fields, float),
                                float(dt), int(n_walkers), int(n_steps), int(mgs_every),
                                int(energy_every), int(seed), int(checkpoint))
