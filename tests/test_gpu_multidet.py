"""Multi-determinant trial on the GPU (afqmc_setup_multidet, FP64) against the oracle at 1e-9:
per-walker weights, log-overlaps with psi_T, determinants and local energies after 50 steps on
the shared field stream, and the correlated pair's per-repeat mixed energies (Sec. II.B with the
truncated CASCI trials standing in for the paper's CASSCF expansions, Sec. II.D)."""
import numpy as np
import pytest

from gpu_util import logo_close, need_gpu, rel, system_data
from oracle import afqmc as orc
from oracle.philox import gaussian_fields
from synthetic import CONFIGS
from synthetic.multidet import cas_trial

pytestmark = pytest.mark.gpu
TOL = 1e-9


def trial_of(d, n_orb, threshold=0.01):
    return cas_trial(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], n_orb,
                     threshold=threshold)


def systems(afq, d, md, nw, dt, seed=1, R=1, mode=0):
    dets, c, start, _ = md
    g = afq.System(d["h1"], d["L"], None, d["n_up"], d["n_dn"], dt=dt, n_walkers=nw, seed=seed,
                   n_repeats=R, mode=mode, dets=dets, coeffs=c, start=start)
    o = orc.System(d["h1"], d["L"], None, d["n_up"], d["n_dn"], dt, dets=dets, coeffs=c,
                   start=start, mode=orc.FREE if mode == 1 else orc.PHASELESS)
    return g, o


def compare(g, wk, el_o=None, el=None, tol=TOL, index=None):
    st = g.state()
    sel = slice(None) if index is None else index
    live = wk.alive
    assert np.array_equal(st["alive"][sel], live)
    np.testing.assert_allclose(st["w"].real[sel], wk.w.real, rtol=tol, atol=0)
    scale = np.abs(wk.phi).max(axis=(1, 2))
    assert (np.abs(st["phi"][sel] - wk.phi).max(axis=(1, 2)) / scale).max() < tol
    assert logo_close(st["logO"][sel][live], wk.logO[live], tol)
    if el is not None:
        assert rel(el[sel][live], el_o[live]) < tol


@pytest.mark.parametrize("which", ["A", "B"])
def test_multidet_walkers_match_oracle_C1(which):
    afq = need_gpu()
    d = system_data("C1", which)
    md = trial_of(d, 6)
    assert len(md[1]) > 10
    nw, seed, dt = 64, 5, CONFIGS["C1"]["dt"]
    g, o = systems(afq, d, md, nw, dt, seed=seed)
    wk = orc.Walkers(o, nw)
    compare(g, wk)                                          # log <psi_T|phi> at the start
    k = np.arange(nw)
    for blk in range(10):
        g.propagate(5)
        for t in range(5 * blk, 5 * blk + 5):
            orc.propagate(o, wk, gaussian_fields(seed, t, k, o.X))
        g.orthonormalise()
        orc.orthonormalise(o, wk)
    el, _, _ = g.energy()
    compare(g, wk, orc.local_energy(o, wk.phi), el)
    g.close()


def test_multidet_full_size_M64_sampled_walkers():
    """The M=64 neutral system (Nchol=320, 8/8) with its CASCI trial over 9 orbitals, 2048
    walkers; the oracle follows sampled pair indices."""
    afq = need_gpu()
    d = system_data("C2", "A", "moderate")
    md = trial_of(d, 9)
    nw, seed, dt, steps = 2048, 2, CONFIGS["C2"]["dt"], 20
    g, o = systems(afq, d, md, nw, dt, seed=seed, R=11)
    sample = np.array([0, 1, 1000, 2047])
    wk = orc.Walkers(o, sample.size)
    for t in range(steps):
        orc.propagate(o, wk, gaussian_fields(seed, t, sample, o.X))
        if (t + 1) % 5 == 0:
            orc.orthonormalise(o, wk)
    for _ in range(steps // 5):
        g.propagate(5)
        g.orthonormalise()
    el, _, _ = g.energy()
    compare(g, wk, orc.local_energy(o, wk.phi), el, index=sample)
    g.close()


def test_multidet_pair_matches_oracle():
    """Correlated pair (neutral 2/2 and ion 2/1), both with multi-determinant trials, through the
    captured pair graph."""
    afq = need_gpu()
    dA, dB = system_data("C1", "A"), system_data("C1", "B")
    nw, R, seed, dt, steps = 48, 3, 7, CONFIGS["C1"]["dt"], 30
    gA, oA = systems(afq, dA, trial_of(dA, 6), nw, dt, seed=seed, R=R)
    gB, oB = systems(afq, dB, trial_of(dB, 6), nw, dt, seed=seed, R=R)
    res = afq.pair_delta_E(gA, gB, steps, 5, 5)
    ref = orc.run_pair(oA, oB, nw, steps, seed=seed, n_repeats=R)
    assert rel(res["E"][:, 0, :], ref["E"][0]) < TOL
    assert rel(res["E"][:, 1, :], ref["E"][1]) < TOL
    gA.close()
    gB.close()


def test_multidet_free_projection_matches_oracle():
    afq = need_gpu()
    d = system_data("C1", "B")
    nw, seed, dt = 32, 3, CONFIGS["C1"]["dt"]
    g, o = systems(afq, d, trial_of(d, 6), nw, dt, seed=seed, mode=1)
    g.propagate(20)
    wk = orc.Walkers(o, nw)
    for t in range(20):
        orc.propagate(o, wk, gaussian_fields(seed, t, np.arange(nw), o.X))
    st = g.state()
    np.testing.assert_allclose(st["w"], wk.w, rtol=TOL, atol=TOL * np.abs(wk.w).max())
    assert logo_close(st["logO"], wk.logO, TOL)
    g.close()


def test_multidet_refusals():
    afq = need_gpu()
    d = system_data("C1", "A")
    dets, c, start, _ = trial_of(d, 6)
    with pytest.raises(afq.AfqmcError, match="invalid argument"):
        afq.System(d["h1"], d["L"], None, 2, 2, dt=0.01, n_walkers=8, dets=dets, coeffs=c,
                   start=start, precision=afq.BF16X3)
    with pytest.raises(afq.AfqmcError, match="invalid argument"):
        afq.System(d["h1"], d["L"], None, 2, 2, dt=0.01, n_walkers=8, dets=dets,
                   coeffs=np.zeros_like(c), start=start)
    g = afq.System(d["h1"], d["L"], None, 2, 2, dt=0.01, n_walkers=8, dets=dets, coeffs=c,
                   start=start)
    with pytest.raises(afq.AfqmcError, match="invalid argument"):
        g.set_tangent(np.eye(d["M"]))
    with pytest.raises(afq.AfqmcError, match="invalid argument"):
        g.adjoint_run(5)
    g.close()
