"""Pins of the oracle's reverse-mode dE/dh1: its contraction with any symmetric P equals the
(separately pinned) tangent-mode dE/dlambda along P, and central differences in one entry."""
import numpy as np
import pytest

from oracle import adjoint, afqmc, tangent
from synthetic import CONFIGS, build_system, explicit_fields


def sym(M, seed, scale=0.01):
    rng = np.random.default_rng(seed)
    P = rng.standard_normal((M, M)) * scale
    return P + P.T


@pytest.mark.parametrize("which,cap", [("A", 1.0), ("B", 1.0), ("A", 0.05)])
def test_gradient_contracts_to_tangent(which, cap):
    d = build_system(**CONFIGS["C1"][which])
    nw, steps = 16, 20
    fields = explicit_fields(steps, nw, d["X"], seed=31)
    s = afqmc.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], 0.01, fb_cap=cap)
    E, G = adjoint.run_with_gradient(s, nw, steps, fields)
    for seed in (1, 2):
        P = sym(d["M"], seed)
        ref, _, _ = tangent.run(s, P, nw, steps, fields)
        assert abs(E - ref[:, 0].mean()) < 1e-12 * abs(E)
        assert abs(np.sum(G * P) - ref[:, 1].mean()) < 1e-8 * max(1.0, abs(ref[:, 1].mean()))


def test_gradient_entry_by_central_differences():
    d = build_system(**CONFIGS["C1"]["B"])
    nw, steps = 16, 10
    fields = explicit_fields(steps, nw, d["X"], seed=32)
    s = afqmc.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], 0.01)
    _, G = adjoint.run_with_gradient(s, nw, steps, fields)
    i, j, eps = 1, 3, 1e-5
    P = np.zeros((d["M"], d["M"]))
    P[i, j] = P[j, i] = 1.0

    def energy(lam):
        sl = afqmc.System(d["h1"] + lam * P, d["L"], d["trial"], d["n_up"], d["n_dn"], 0.01)
        return adjoint.run_with_gradient(sl, nw, steps, fields)[0]

    fd = (energy(eps) - energy(-eps)) / (2 * eps)
    assert abs(G[i, j] + G[j, i] - fd) < 1e-6 * max(1.0, abs(fd))
