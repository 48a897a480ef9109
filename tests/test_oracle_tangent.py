"""Pins of the oracle's tangent-mode derivative dE/dlambda (h1 -> h1 + lambda P) against
central finite differences under common random numbers (same explicit fields)."""
import numpy as np
import pytest

from oracle import afqmc, tangent
from synthetic import CONFIGS, build_system, explicit_fields


def perturbation(M, seed=3, scale=0.01):
    rng = np.random.default_rng(seed)
    P = rng.standard_normal((M, M)) * scale
    return P + P.T


def energies(d, lam, P, nw, steps, fields, dt=0.01, fb_cap=1.0):
    s = afqmc.System(d["h1"] + lam * P, d["L"], d["trial"], d["n_up"], d["n_dn"], dt, fb_cap=fb_cap)
    out, _, _ = tangent.run(s, P, nw, steps, fields)
    return out


def test_frechet_derivative_of_exp():
    rng = np.random.default_rng(1)
    B = rng.standard_normal((5, 5)) * 0.1
    B = B + B.T
    dB = rng.standard_normal((5, 5))
    dB = dB + dB.T
    from scipy.linalg import expm
    _, F = tangent.frechet_exp(B, dB)
    eps = 1e-6
    fd = (expm(B + eps * dB) - expm(B - eps * dB)) / (2 * eps)
    np.testing.assert_allclose(F, fd, atol=1e-9)


@pytest.mark.parametrize("which,cap", [("A", 1.0), ("B", 1.0), ("A", 0.05)])
def test_tangent_matches_central_differences(which, cap):
    d = build_system(**CONFIGS["C1"][which])
    nw, steps = 32, 20
    fields = explicit_fields(steps, nw, d["X"], seed=12)
    P = perturbation(d["M"])
    base = energies(d, 0.0, P, nw, steps, fields, fb_cap=cap)
    eps = 1e-5
    ep = energies(d, eps, P, nw, steps, fields, fb_cap=cap)
    em = energies(d, -eps, P, nw, steps, fields, fb_cap=cap)
    fd = (ep[:, 0] - em[:, 0]) / (2 * eps)
    np.testing.assert_allclose(base[:, 1], fd, rtol=2e-5, atol=2e-7)
    assert np.all(np.abs(base[:, 1]) > 1e-4)      # a real derivative, not a trivial zero


def test_tangent_of_trial_energy_and_one_body_term():
    """At tau = 0 (walkers = trial) dE/dlambda = tr(P P_trial) exactly."""
    d = build_system(**CONFIGS["C1"]["A"])
    s = afqmc.System(d["h1"], d["L"], d["trial"], 2, 2, 0.01)
    P = perturbation(d["M"])
    ts = tangent.TangentSystem(s, P)
    phi = np.broadcast_to(d["trial"], (3, d["M"], 4)).astype(complex)
    e, de = tangent.local_energy_tangent(ts, phi, np.zeros_like(phi))
    assert np.allclose(de, ts.dE_T)
