"""Correlated free projection through the pair graph (the paper's correlated
free-projection comparison): both systems with x_bar = 0 and complex weights, no cos cut,
E = Re(sum w E_L / sum w) per repeat. FP64 path against the oracle's run_pair in free mode at
1e-9."""
import numpy as np
import pytest

from gpu_util import need_gpu, pair, rel, system_data
from oracle import afqmc as orc
from synthetic import CONFIGS

pytestmark = pytest.mark.gpu
TOL = 1e-9


def test_free_projection_pair_graph_matches_oracle():
    afq = need_gpu()
    cfg = CONFIGS["C1"]
    dA, dB = system_data("C1", "A"), system_data("C1", "B")
    nw, R, seed, steps = 64, 4, 23, 30
    gA, oA = pair(afq, dA, nw, cfg["dt"], seed=seed, R=R, mode=1)
    gB, oB = pair(afq, dB, nw, cfg["dt"], seed=seed, R=R, mode=1)
    res = afq.pair_delta_E(gA, gB, steps, energy_every=5, mgs_every=5, tau_eq=0.05)
    ref = orc.run_pair(oA, oB, nw, steps, seed=seed, n_repeats=R)
    assert rel(res["E"][:, 0, :], ref["E"][0]) < TOL
    assert rel(res["E"][:, 1, :], ref["E"][1]) < TOL
    wkA, wkB = ref["walkers"]
    for g, wk in ((gA, wkA), (gB, wkB)):
        st = g.state()
        assert np.all(st["alive"])                          # no phaseless cut in free mode
        np.testing.assert_allclose(st["w"], wk.w, rtol=TOL, atol=TOL * np.abs(wk.w).max())
    assert np.abs(wkA.w.imag).max() > 1e-6                  # complex weights really exercised
    gA.close()
    gB.close()
