"""Preliminary equilibration scheme on the GPU (Sec. II.C) against the oracle (FP64, 1e-9):
the comb of the primary system per repeat (the same walker indices: an index mismatch shows
as an O(1) difference), the seeding of an ion from the neutral, and the correlated run that
follows.
"""
import numpy as np
import pytest

from gpu_util import logo_close, need_gpu, pair, rel, system_data
from oracle import afqmc as orc
from oracle import pes
from oracle.philox import gaussian_fields
from synthetic import CONFIGS

pytestmark = pytest.mark.gpu
TOL = 1e-9


def compare(g, wk, tol=TOL):
    st = g.state()
    assert np.array_equal(st["alive"], wk.alive)
    np.testing.assert_allclose(st["w"].real, wk.w.real, rtol=tol, atol=0)
    scale = np.abs(wk.phi).max(axis=(1, 2))
    assert (np.abs(st["phi"] - wk.phi).max(axis=(1, 2)) / scale).max() < tol
    assert logo_close(st["logO"][wk.alive], wk.logO[wk.alive], tol)


def equilibrate(afq, g, o, nw, R, seed, u, blocks):
    """Both sides: [5 steps, MGS, comb] x blocks on the internal field stream."""
    wk = orc.Walkers(o, nw)
    groups = orc.repeat_groups(nw, R)
    t = 0
    for b in range(blocks):
        g.propagate(5)
        for _ in range(5):
            orc.propagate(o, wk, gaussian_fields(seed, t, np.arange(nw), o.X))
            t += 1
        g.orthonormalise()
        orc.orthonormalise(o, wk)
        g.population_control(u[b])
        pes.population_control(o, wk, groups, R, u[b])
        compare(g, wk)
    return wk


def test_population_control_matches_oracle():
    afq = need_gpu()
    d = system_data("C1", "A")
    nw, R, seed = 24, 3, 41
    g, o = pair(afq, d, nw, CONFIGS["C1"]["dt"], seed=seed, R=R)
    u = np.array([[0.31, 0.72, 0.05], [0.5, 0.999, 0.2]])
    wk = equilibrate(afq, g, o, nw, R, seed, u, 2)
    g.propagate(5)                        # the combed population propagates on
    for t in range(10, 15):
        orc.propagate(o, wk, gaussian_fields(seed, t, np.arange(nw), o.X))
    compare(g, wk)
    g.close()


def test_seeding_and_correlated_run_match_oracle():
    afq = need_gpu()
    cfg = CONFIGS["C1"]
    # neutral 2/2, ion 2/1 at the moderate coupling: there the two SCF trials share their
    # orbitals (overlaps 0.97-0.98), so a walker of the neutral seeds the ion with R > 0; at the
    # literal coupling the ion's trial is rotated far from the neutral's and R < 0 for every
    # walker, which the phaseless projection of the seeding kills
    dA, dB = system_data("C1", "A", "moderate"), system_data("C1", "B", "moderate")
    nw, R, seed, n_eq, n_steps = 32, 2, 43, 10, 20
    u = np.array([[0.25, 0.75], [0.6, 0.1]])
    gA, oA = pair(afq, dA, nw, cfg["dt"], seed=seed, R=R)
    gB, oB = pair(afq, dB, nw, cfg["dt"], seed=seed, R=R)
    wkA = equilibrate(afq, gA, oA, nw, R, seed, u, n_eq // 5)
    gB.seed_from(gA)
    assert gB.info().step == n_eq
    compare(gB, pes.seed_secondary(oA, oB, wkA))
    res = afq.pair_delta_E(gA, gB, n_steps, 5, 5)
    ref = pes.run_pes(oA, oB, nw, n_eq, n_steps, seed, u, n_repeats=R)
    assert rel(res["E"][:, 0, :], ref["E"][0]) < TOL
    assert rel(res["E"][:, 1, :], ref["E"][1]) < TOL
    gA.close()
    gB.close()


def test_population_control_refusals():
    afq = need_gpu()
    d = system_data("C1", "A")
    g, _ = pair(afq, d, 8, 0.01, R=2)
    with pytest.raises(ValueError):
        g.population_control([0.5])                                # one uniform per repeat
    w = np.ones(8)
    w[:4] = 0.0                                                    # repeat 0 has no live walker
    phi = g.state()["phi"]
    g.set_walkers(phi, w)
    with pytest.raises(afq.AfqmcError, match="numerical"):
        g.population_control([0.5, 0.5])
    assert np.array_equal(g.state()["w"].real, w)                   # left unchanged
    f, _ = pair(afq, d, 8, 0.01, R=2, mode=1)
    with pytest.raises(afq.AfqmcError, match="invalid argument"):
        f.population_control([0.5, 0.5])                          # free projection: refused
    dB = system_data("C1", "B")
    ion, _ = pair(afq, dB, 8, 0.01, R=2)
    with pytest.raises(afq.AfqmcError, match="invalid argument"):
        g.seed_from(ion)                                           # more electrons than primary
    for h in (g, f, ion):
        h.close()
