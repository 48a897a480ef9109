"""Reverse mode on the GPU: dE/dh1 of one run's mixed energy by the checkpointed adjoint.

Checked element by element against the oracle's reverse pass (itself pinned against the
tangent and by central differences), including a run in which walkers die and the force
bias is capped; for invariance under the checkpoint interval (every recomputation replays
the forward pass exactly); against the GPU tangent mode at the C5 shape (M=96, Nchol=480,
12/12) on the Philox stream; and for the handle's state after the call.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, system_data
from oracle import adjoint as oadj
from oracle import afqmc as orc
from synthetic import CONFIGS, explicit_fields

pytestmark = pytest.mark.gpu


def sym(M, seed, scale=0.01):
    rng = np.random.default_rng(seed)
    P = rng.standard_normal((M, M)) * scale
    return P + P.T


def gpu_system(afq, d, nw, dt, fb_cap=1.0, seed=1):
    return afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=dt, n_walkers=nw,
                      seed=seed, fb_cap=fb_cap)


@pytest.mark.parametrize("which,dt,cap,steps,ee,me", [
    ("A", 0.01, 1.0, 20, 5, 5),
    ("B", 0.01, 1.0, 23, 5, 5),     # spin-unbalanced; last three steps after the final measurement
    ("A", 0.1, 0.3, 20, 5, 5),      # 5 of 16 walkers die, the cap is active
    ("B", 0.05, 1.0, 12, 3, 4),     # measurement and Gram-Schmidt intervals differ
])
def test_adjoint_matches_oracle(which, dt, cap, steps, ee, me):
    afq = need_gpu()
    d = system_data("C1", which)
    nw = 16
    fields = explicit_fields(steps, nw, d["X"], seed=41)
    o = orc.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt, fb_cap=cap)
    E_ref, G_ref = oadj.run_with_gradient(o, nw, steps, fields, mgs_every=me, energy_every=ee)
    s = gpu_system(afq, d, nw, dt, fb_cap=cap)
    E, G = s.adjoint_run(steps, fields, mgs_every=me, energy_every=ee, checkpoint=4)
    s.close()
    assert abs(E - E_ref) < 1e-10 * abs(E_ref)
    scale = np.abs(G_ref).max()
    np.testing.assert_allclose(G, G_ref, rtol=1e-7, atol=1e-9 * scale)


def test_checkpoint_interval_does_not_change_the_result():
    afq = need_gpu()
    d = system_data("C1", "A")
    nw, steps, dt = 16, 20, 0.1
    fields = explicit_fields(steps, nw, d["X"], seed=41)
    out = []
    for K in (1, 3, 7, 20, 50):
        s = gpu_system(afq, d, nw, dt, fb_cap=0.3)
        out.append(s.adjoint_run(steps, fields, checkpoint=K))
        s.close()
    for E, G in out[1:]:
        assert E == out[0][0]
        assert np.array_equal(G, out[0][1])


def test_handle_ends_after_the_run():
    afq = need_gpu()
    d = system_data("C1", "B")
    nw, steps, dt = 16, 13, 0.01
    a = gpu_system(afq, d, nw, dt)
    b = gpu_system(afq, d, nw, dt)
    a.adjoint_run(steps, None, mgs_every=5, energy_every=5, checkpoint=4)
    for t in range(steps):
        b.propagate(1)
        if (t + 1) % 5 == 0:
            b.orthonormalise()
    sa, sb = a.state(), b.state()
    assert np.array_equal(sa["phi"], sb["phi"])
    assert np.array_equal(sa["w"], sb["w"])
    # the next Philox step continues the stream where a plain run would
    a.propagate(2)
    b.propagate(2)
    assert np.array_equal(a.state()["phi"], b.state()["phi"])
    a.close()
    b.close()


def test_adjoint_contracts_to_gpu_tangent_C5_shape():
    afq = need_gpu()
    d = system_data("C5", "A", "moderate")
    nw, steps, dt = 128, 20, CONFIGS["C5"]["dt"]
    s = gpu_system(afq, d, nw, dt)
    E, G = s.adjoint_run(steps, None, mgs_every=5, energy_every=5, checkpoint=5)
    s.close()
    for seed in (5, 6):
        P = sym(d["M"], seed)
        t = gpu_system(afq, d, nw, dt)
        t.set_tangent(P)
        es, ds = [], []
        for blk in range(steps // 5):
            t.propagate(5)
            t.orthonormalise()
            em, dm, _ = t.energy_tangent()
            es.append(em[0])
            ds.append(dm[0])
        t.close()
        assert abs(E - np.mean(es)) < 1e-11 * abs(E)
        ref = np.mean(ds)
        assert abs(np.sum(G * P) - ref) < 1e-7 * max(abs(ref), np.sum(np.abs(G * P)))


def test_adjoint_argument_errors():
    afq = need_gpu()
    d = system_data("C1", "A")
    s = gpu_system(afq, d, 8, 0.01)
    with pytest.raises(RuntimeError):
        s.adjoint_run(10, None, energy_every=11)
    with pytest.raises(RuntimeError):
        s.adjoint_run(0, None)
    s.set_tangent(sym(d["M"], 1))
    with pytest.raises(RuntimeError):
        s.adjoint_run(10, None)
    s.close()
    m = afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=0.01, n_walkers=8,
                   precision=afq.BF16X3)
    with pytest.raises(RuntimeError):
        m.adjoint_run(10, None)
    m.close()


def test_autograd_h1_gradient_matches_tangent_runs():
    """One reverse sweep gives the gradient that M(M+1)/2 tangent runs give, entry by entry."""
    afq = need_gpu()
    import torch
    from paper_1703_01545_gb300.autograd import mixed_energy_grad_h1, mixed_energy_h1
    d = system_data("C1", "B")
    nw, steps = 16, 10
    fields = explicit_fields(steps, nw, d["X"], seed=4)
    h1 = torch.tensor(d["h1"], dtype=torch.float64, requires_grad=True)
    E = mixed_energy_h1(h1, d["L"], d["trial"], d["n_up"], d["n_dn"], fields=fields,
                        n_walkers=nw, n_steps=steps, checkpoint=3)
    (g,) = torch.autograd.grad(E, h1)
    g = g.numpy()
    G_tan = mixed_energy_grad_h1(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"],
                                 fields=fields, n_walkers=nw, n_steps=steps)
    np.testing.assert_allclose(0.5 * (g + g.T), G_tan, rtol=1e-7, atol=1e-9 * np.abs(G_tan).max())
    o = orc.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], 0.01)
    E_ref, _ = oadj.run_with_gradient(o, nw, steps, fields)
    assert abs(float(E.detach()) - E_ref) < 1e-10 * abs(E_ref)
