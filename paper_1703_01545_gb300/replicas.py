"""Replicas of the correlated pair on several GPUs, one process per GPU.

Without population control every pair index k evolves on its own (Sec. II.B), so N processes
split the pair indices into disjoint ranges and exchange nothing while they propagate. Rank r
takes k in [r Nw, (r+1) Nw) through ``walker_offset``, draws for each k the same fields a single
process would, and forms its own R repeats from its walkers. After the run the per-repeat
energy series are gathered, and the Delta E statistics of Sec. II.B are taken over all N R
repeats. The gather is host-side ``torch.distributed`` (gloo, or NCCL with the series on the
rank's current CUDA device); the statistics are the library's host routine.
"""
import numpy as np


def walker_offset(rank: int, n_walkers: int) -> int:
    """Global pair index of the first walker of ``rank`` when every rank holds n_walkers."""
    if rank < 0 or n_walkers < 1:
        raise ValueError("need rank >= 0 and n_walkers >= 1")
    return rank * n_walkers


def gather_series(E, group=None):
    """Collective over ``group`` (every rank calls it; every rank gets the result): the
    per-repeat energy series E [n_meas, 2, R] of all ranks as [n_meas, 2, world * R], rank r's
    repeat j in column r * R + j. Every rank must pass the same shape."""
    import torch
    import torch.distributed as dist

    t = torch.from_numpy(np.ascontiguousarray(E, dtype=np.float64))
    if "nccl" in str(dist.get_backend(group)):
        t = t.cuda()
    parts = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, t, group=group)
    return np.concatenate([p.cpu().numpy() for p in parts], axis=2)


def merged_delta_E(E_all, taus, tau_eq):
    """(mean, standard error, tau at the earliest minimum error) of Delta E = E_B - E_A over
    all repeats of E_all [n_meas, 2, R_total]: the cumulative averages after tau_eq, as the
    pair call reports them for one process."""
    from .api import afqmc_delta_E_stats

    E_all = np.asarray(E_all, dtype=np.float64)
    dE = E_all[:, 1, :] - E_all[:, 0, :]
    _, _, est = afqmc_delta_E_stats(dE, np.asarray(taus, dtype=np.float64), tau_eq)
    return est
