"""Fault injection on the host (no GPU fault): walkers handed over with an exactly singular
overlap (a zero column) or a non-finite entry are killed (w = 0, not alive) by the overlap
kernel and counted, the others are untouched, the mixed estimate stays finite, and the run
continues with the dead walkers frozen."""
import numpy as np
import pytest

from gpu_util import need_gpu, system_data

pytestmark = pytest.mark.gpu


def test_singular_and_non_finite_walkers_are_killed_without_poisoning_the_estimate():
    afq = need_gpu()
    d = system_data("C1", "A")
    nw = 8
    g = afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=0.01, n_walkers=nw,
                   seed=3)
    rng = np.random.default_rng(4)
    phi = d["trial"][None] + 0.05 * (rng.standard_normal((nw,) + d["trial"].shape) +
                                     1j * rng.standard_normal((nw,) + d["trial"].shape))
    phi[3][:, 0] = 0.0            # a zero column: the spin-up overlap is exactly singular
    phi[5][0, 1] = np.nan         # a non-finite entry
    g.set_walkers(phi)
    st = g.state()
    dead = np.zeros(nw, bool)
    dead[[3, 5]] = True
    assert np.array_equal(st["alive"], ~dead)
    assert np.all(st["w"][dead] == 0) and np.all(st["w"].real[~dead] == 1.0)
    _, em, ws = g.energy()
    assert np.isfinite(em[0]) and ws[0] == nw - 2
    g.propagate(5)
    g.orthonormalise()
    st2 = g.state()
    assert not st2["alive"][dead].any()                        # dead for good
    assert np.all(np.isfinite(st2["w"].real)) and np.all(st2["w"][dead] == 0)
    _, em2, _ = g.energy()
    assert np.isfinite(em2[0])
    g.close()
