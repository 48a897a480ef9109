"""Rank body of the two-process gloo test of the replica path (spawned, top-level so that
the child processes can import it)."""
import os

import numpy as np


def shard_series(rank, world, nw, R, steps, seed):
    """Rank's per-repeat series [n_meas, 2, R] for pair indices [rank nw, (rank + 1) nw): the
    oracle run on that range, its repeats formed from its own walkers (walker i of the rank in
    repeat i R / nw) as a handle with walker_offset = rank nw forms them."""
    from oracle import afqmc as orc
    from paper_1703_01545_gb300.replicas import walker_offset
    from synthetic import CONFIGS, build_system

    sA, sB = (orc.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], CONFIGS["C1"]["dt"])
              for d in (build_system(**CONFIGS["C1"][w]) for w in ("A", "B")))
    k = walker_offset(rank, nw) + np.arange(nw)
    # global population world * nw with world * R repeats: rank r's walkers fall in repeats
    # r R + (i R) / nw, the rank's own R repeats in order
    r = orc.run_pair(sA, sB, world * nw, steps, seed=seed, n_repeats=world * R, walker_index=k)
    cols = slice(rank * R, (rank + 1) * R)
    return np.stack([r["E"][0][:, cols], r["E"][1][:, cols]], axis=1), np.array(r["steps"])


def run(rank, world, port, out_dir, nw, R, steps, seed, tau_eq):
    import torch.distributed as dist
    from paper_1703_01545_gb300.replicas import gather_series, merged_delta_E
    from synthetic import CONFIGS

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        E, steps_done = shard_series(rank, world, nw, R, steps, seed)
        E_all = gather_series(E)
        taus = steps_done * CONFIGS["C1"]["dt"]
        est = merged_delta_E(E_all, taus, tau_eq)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), E=E, E_all=E_all, est=np.array(est))
        dist.barrier()
    finally:
        dist.destroy_process_group()
