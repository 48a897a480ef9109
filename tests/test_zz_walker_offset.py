"""walker_offset on the GPU: walker i of a handle with walker_offset = K draws the fields of
pair index K + i. That is the layout of replicas on several GPUs, each rank holding its own
range of pair indices. The FP64 path is held to the oracle at 1e-9; the split path's field
kernel forms the same counter (K + i, t, g)."""
import numpy as np
import pytest

from gpu_util import logo_close, need_gpu, rel, system_data
from oracle import afqmc as orc
from oracle.philox import gaussian_fields

pytestmark = pytest.mark.gpu
TOL = 1e-9


def test_walker_offset_draws_the_fields_of_its_pair_indices():
    afq = need_gpu()
    d = system_data("C1", "A")
    nw, K, seed, dt = 24, 1000, 31, 0.01

    def handle(offset):
        return afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=dt,
                          n_walkers=nw, seed=seed, walker_offset=offset)

    g, g0 = handle(K), handle(0)
    o = orc.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt)
    wk = orc.Walkers(o, nw)
    k = K + np.arange(nw)
    t = 0
    for _ in range(2):
        for h in (g, g0):
            h.propagate(5)
            h.orthonormalise()
        for _ in range(5):
            orc.propagate(o, wk, gaussian_fields(seed, t, k, o.X))
            t += 1
        orc.orthonormalise(o, wk)
    st = g.state()
    assert np.array_equal(st["alive"], wk.alive)
    np.testing.assert_allclose(st["w"].real, wk.w.real, rtol=TOL, atol=0)
    scale = np.abs(wk.phi).max(axis=(1, 2))
    assert (np.abs(st["phi"] - wk.phi).max(axis=(1, 2)) / scale).max() < TOL
    assert logo_close(st["logO"][wk.alive], wk.logO[wk.alive], TOL)
    el, _, _ = g.energy()
    assert rel(el, orc.local_energy(o, wk.phi)) < TOL
    # the offset is really applied: pair indices 0..nw-1 walk elsewhere
    assert np.abs(g0.state()["phi"] - st["phi"]).max() > 1e-3
    g.close()
    g0.close()
