"""The replica path on CPU: two gloo ranks, each on its own range of pair indices, gather
their per-repeat energy series and merge the Delta E statistics; the result must be that of
one population over all pair indices (the shards exchange nothing while they propagate,
Sec. II.B)."""
import socket

import numpy as np
import pytest

from oracle import afqmc as orc
from oracle import stats
from synthetic import CONFIGS, build_system


def free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_walker_offsets_partition_the_pair_indices():
    from paper_1703_01545_gb300.replicas import walker_offset
    world, nw = 4, 37
    ranges = [set(range(walker_offset(r, nw), walker_offset(r, nw) + nw)) for r in range(world)]
    assert set().union(*ranges) == set(range(world * nw))
    assert sum(len(x) for x in ranges) == world * nw
    with pytest.raises(ValueError):
        walker_offset(-1, nw)


def test_two_gloo_ranks_merge_to_the_single_population(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    from paper_1703_01545_gb300.build import build
    import replica_worker

    build()   # the host statistics live in the library
    world, nw, R, steps, seed, tau_eq = 2, 12, 3, 20, 17, 0.05
    mp.spawn(replica_worker.run, args=(world, free_port(), str(tmp_path), nw, R, steps, seed,
                                       tau_eq), nprocs=world, join=True)
    got = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]

    # one process over all world * nw pair indices with world * R repeats
    sA, sB = (orc.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], CONFIGS["C1"]["dt"])
              for d in (build_system(**CONFIGS["C1"][w]) for w in ("A", "B")))
    ref = orc.run_pair(sA, sB, world * nw, steps, seed=seed, n_repeats=world * R)
    E_ref = np.stack([ref["E"][0], ref["E"][1]], axis=1)
    for r in range(world):
        assert np.array_equal(got[r]["E"], E_ref[:, :, r * R:(r + 1) * R])
        assert np.array_equal(got[r]["E_all"], E_ref)            # every rank gets the gather
    taus = np.array(ref["steps"]) * CONFIGS["C1"]["dt"]
    m, s, t = stats.delta_e_estimate(ref["E"][1] - ref["E"][0], taus, tau_eq)
    for r in range(world):
        np.testing.assert_allclose(got[r]["est"], [m, s, t], rtol=1e-12, atol=1e-15)
