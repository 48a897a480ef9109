"""Uneven correlated pair (A: M=200, Nchol=1000, 9/9; B: M=190, Nchol=950, 8/8, its own
Hamiltonian from seed 2703), full size (2048 walkers per system), both precisions.

Walker k of B draws the first 950 of the fields that walker k of A draws (the stream
depends on (seed, step, k, g) only).  The oracle follows sampled pair indices exactly.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, system_data
from oracle import afqmc as orc
from synthetic import CONFIGS

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,taylor", [("fp64", None), ("bf16x3", None), ("bf16x3", 4)])
def test_uneven_pair_full_size_sampled_walkers(precision, taylor):
    """taylor: the propagation variant forced on both systems (4: the tensor-core propagator
    over streamed split-BF16 V_HS), or the autotuner's choice."""
    afq = need_gpu()
    cfg = CONFIGS["C4"]
    nw, dt, steps = cfg["n_walkers"], cfg["dt"], 10
    prec = afq.FP64 if precision == "fp64" else afq.BF16X3
    # split path: ten times the per-walker error measured at the M=64 shapes (w ~1e-4)
    tol_w, tol_phi = (1e-9, 1e-9) if precision == "fp64" else (1e-3, 1e-3)
    data = [system_data("C4", w, "moderate") for w in ("A", "B")]
    gpu = [afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=dt, n_walkers=nw,
                      seed=3, n_repeats=11, precision=prec) for d in data]
    if taylor is not None:
        for g in gpu:
            g.select_kernel(afq.K_TAYLOR, taylor)
    res = afq.pair_delta_E(gpu[0], gpu[1], steps, 5, 5)
    assert np.all(np.isfinite(res["E"]))
    sample = np.array([0, 777, 2047])
    osys = [orc.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt) for d in data]
    ref = orc.run_pair(osys[0], osys[1], nw, steps, seed=3, energy_every=0, mgs_every=5,
                       walker_index=sample)
    for g, wk in zip(gpu, ref["walkers"]):
        st = g.state()
        assert np.array_equal(st["alive"][sample], wk.alive)
        np.testing.assert_allclose(st["w"].real[sample], wk.w.real, rtol=tol_w, atol=0)
        err = np.abs(st["phi"][sample] - wk.phi).max() / np.abs(wk.phi).max()
        assert err < tol_phi, err
        d = np.exp(st["logO"][sample] - wk.logO) - 1
        assert np.abs(d).max() < tol_w
    for g in gpu:
        g.close()
