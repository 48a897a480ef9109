"""Tangent mode on the GPU: dE/dlambda along h1 -> h1 + lambda P on a fixed field realisation.

Checked against the oracle's tangent (itself pinned by central differences), against
central differences of GPU runs at h1 +- eps P on the same fields (the C5 shape: M=96,
Nchol=480, 12/12), and through the torch.autograd wrapper.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, system_data
from oracle import afqmc as orc
from oracle import tangent as otan
from synthetic import CONFIGS, explicit_fields

pytestmark = pytest.mark.gpu


def perturbation(M, seed=3, scale=0.01):
    rng = np.random.default_rng(seed)
    P = rng.standard_normal((M, M)) * scale
    return P + P.T


def gpu_tangent_run(afq, d, P, nw, steps, fields, dt, lam=0.0):
    s = afq.System(d["h1"] + lam * P, d["L"], d["trial"], d["n_up"], d["n_dn"], dt=dt, n_walkers=nw)
    s.set_tangent(P)
    out = []
    for blk in range(steps // 5):
        s.propagate(5, fields[5 * blk:5 * blk + 5])
        s.orthonormalise()
        em, dm, _ = s.energy_tangent()
        out.append((em[0], dm[0]))
    dlogw = s.tangent_state()
    st = s.state()
    s.close()
    return np.array(out), dlogw, st


@pytest.mark.parametrize("which", ["A", "B"])
def test_tangent_matches_oracle(which):
    afq = need_gpu()
    d = system_data("C1", which)
    nw, steps, dt = 32, 20, 0.01
    fields = explicit_fields(steps, nw, d["X"], seed=12)
    P = perturbation(d["M"])
    got, dlogw, st = gpu_tangent_run(afq, d, P, nw, steps, fields, dt)
    o = orc.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt)
    ref, wk, tw = otan.run(o, P, nw, steps, fields)
    np.testing.assert_allclose(got[:, 0], ref[:, 0], rtol=1e-9)
    np.testing.assert_allclose(got[:, 1], ref[:, 1], rtol=1e-7, atol=1e-9 * np.abs(ref[:, 1]).max())
    np.testing.assert_allclose(dlogw, tw.dlogw, rtol=1e-7, atol=1e-9 * np.abs(tw.dlogw).max())
    np.testing.assert_allclose(st["w"].real, wk.w.real, rtol=1e-9)


def test_tangent_matches_gpu_central_differences_C5_shape():
    afq = need_gpu()
    d = system_data("C5", "A", "moderate")
    nw, steps, dt = 128, 20, CONFIGS["C5"]["dt"]
    fields = explicit_fields(steps, nw, d["X"], seed=21)
    P = perturbation(d["M"], seed=5)
    base, _, _ = gpu_tangent_run(afq, d, P, nw, steps, fields, dt)
    eps = 1e-4
    plus, _, _ = gpu_tangent_run(afq, d, P, nw, steps, fields, dt, lam=eps)
    minus, _, _ = gpu_tangent_run(afq, d, P, nw, steps, fields, dt, lam=-eps)
    fd = (plus[:, 0] - minus[:, 0]) / (2 * eps)
    np.testing.assert_allclose(base[:, 1], fd, rtol=1e-4, atol=1e-6)
    assert np.all(np.abs(base[:, 1]) > 1e-3)


def test_autograd_wrapper_gives_the_tangent():
    afq = need_gpu()
    import torch
    from paper_1703_01545_gb300.autograd import mixed_energy
    d = system_data("C1", "A")
    nw, steps = 32, 20
    fields = explicit_fields(steps, nw, d["X"], seed=12)
    P = perturbation(d["M"])
    lam = torch.tensor(0.0, dtype=torch.float64, requires_grad=True)
    E = mixed_energy(lam, d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], P, fields=fields,
                     n_walkers=nw, n_steps=steps)
    (g,) = torch.autograd.grad(E, lam)
    o = orc.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], 0.01)
    ref, _, _ = otan.run(o, P, nw, steps, fields)
    assert abs(float(E.detach()) - ref[:, 0].mean()) < 1e-9 * abs(ref[:, 0].mean())
    assert abs(float(g) - ref[:, 1].mean()) < 1e-7 * abs(ref[:, 1].mean())


def test_full_gradient_contracts_to_the_directional_derivative():
    """sum_ij (dE/dh1)_ij P_ij equals dE/dlambda along P (linearity of the tangent)."""
    afq = need_gpu()
    from paper_1703_01545_gb300.autograd import mixed_energy_grad_h1
    d = system_data("C1", "B")
    nw, steps = 16, 10
    fields = explicit_fields(steps, nw, d["X"], seed=4)
    G = mixed_energy_grad_h1(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], fields=fields,
                             n_walkers=nw, n_steps=steps)
    np.testing.assert_allclose(G, G.T, atol=0)
    P = perturbation(d["M"], seed=9)
    o = orc.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], 0.01)
    ref, _, _ = otan.run(o, P, nw, steps, fields)
    assert abs(np.sum(G * P) - ref[:, 1].mean()) < 1e-8 * max(1.0, abs(ref[:, 1].mean()))
