"""Planted mistakes in the oracle, each of which must fail at least one of its pins.

Every mutant below is a plausible slip in writing the method down: a sign, a dropped term
or factor, a transposed operand, a conjugation the paper does not have, an off-by-one
order, a stale quantity after orthonormalisation. The mutant replaces one oracle function
(module attribute, so the oracle's internal calls see it too), then the pins of
test_oracle_pins.py and test_oracle_rng.py run cheapest first until one fails. The control
case (no mutant) must pass them all, so the failures come from the mutants.
"""
import numpy as np
import pytest

import test_oracle_pes as PES
import test_oracle_pins as P
import test_oracle_rng as RNG
import test_oracle_stats as ST
from oracle import afqmc, pes, philox, stats

ORIG = {n: getattr(afqmc, n) for n in ("force_bias", "green", "local_energy", "taylor_apply",
                                       "step_determinant", "orthonormalise", "propagate",
                                       "overlap", "modified_gram_schmidt")}
ORIG_INIT = afqmc.System.__init__
ORIG_PES = {n: getattr(pes, n) for n in ("comb_select", "seed_secondary", "seed_columns")}
ORIG_STATS = {n: getattr(stats, n) for n in ("per_tau", "cumulative")}
ORIG_BOX_MULLER = philox.box_muller

PINS = [
    ("overlap vs determinant expansion", lambda: P.test_overlap_is_many_body_overlap(2, 1)),
    ("G as log-overlap derivative", lambda: P.test_green_function_is_log_overlap_derivative(2, 1)),
    ("G invariants", P.test_green_function_invariants),
    ("rhobar as log-overlap derivative", P.test_force_bias_is_log_overlap_derivative),
    ("E_L vs FCI mixed estimate", lambda: P.test_local_energy_is_mixed_estimate_in_fci_space(2, 1)),
    ("E_T vs HF", lambda: P.test_trial_energy_is_hartree_fock_energy(2, 1)),
    ("one electron", P.test_one_electron_has_no_two_body_energy),
    ("Taylor bound", P.test_taylor_error_bound),
    ("MGS", lambda: P.test_modified_gram_schmidt(2, 2)),
    ("Eq. 8 stationarity", P.test_force_bias_is_stationary_point_of_weight),
    # after stationarity: its check of the capped values recomputes the uncapped bias itself
    ("force-bias cap", P.test_force_bias_cap),
    ("non-interacting closed form", P.test_non_interacting_limit_is_deterministic_closed_form),
    ("normal moments", RNG.test_normal_moments),
    ("quadrature, no shift", lambda: P.test_hs_propagator_and_force_bias_by_quadrature(0.0)),
    ("quadrature, complex shift",
     lambda: P.test_hs_propagator_and_force_bias_by_quadrature(0.4 - 0.7j)),
    ("walker death", P.test_walker_death_is_permanent_and_freezes_determinant),
    ("comb weight and dead walkers", PES.test_comb_keeps_the_total_weight_and_skips_dead_walkers),
    ("comb expected copies", PES.test_comb_expected_copies_are_the_weight_shares),
    ("comb within repeats", PES.test_population_control_stays_within_each_repeat),
    ("seeding keeps the state", lambda: PES.test_seeding_keeps_the_represented_state(2)),
    ("seeding an ion", lambda: PES.test_seeding_keeps_the_represented_state(1)),
    ("seeding phase projection", PES.test_seeding_projects_the_phase_of_the_ratio),
    ("repeat mean and error", ST.test_per_tau_mean_and_standard_error),
    ("cumulative averages, earliest minimum", ST.test_cumulative_and_earliest_minimum),
]


def _reinit(after):
    """System.__init__ followed by `after(self)` (a slip in the derived one-body data)."""
    def init(self, *a, **kw):
        ORIG_INIT(self, *a, **kw)
        after(self)
    return init


def _half_step(s, K):
    lam, U = np.linalg.eigh(K)
    return (U * np.exp(-0.5 * s.dt * lam)) @ U.T


def _k_without_LL(s):
    s.K = s.K + 0.5 * np.einsum("gik,gkj->ij", s.L, s.L)
    s.expK = _half_step(s, s.K)


def _k_mean_field_sign(s):
    s.K = s.K - 2 * np.einsum("g,gij->ij", s.rho_mf, s.L)
    s.expK = _half_step(s, s.K)


def _full_step(s):
    lam, U = np.linalg.eigh(s.K)
    s.expK = (U * np.exp(-s.dt * lam)) @ U.T


def _fb_no_mean_field(sys, G):
    saved = sys.rho_mf
    sys.rho_mf = np.zeros_like(saved)
    try:
        return ORIG["force_bias"](sys, G)
    finally:
        sys.rho_mf = saved


def _fb_cap_componentwise(sys, G):
    cap = sys.fb_cap
    raw = -1j * sys.sqrt_dt * (afqmc.rhobar(sys, G) - sys.rho_mf[None, :])
    if cap <= 0:
        return raw
    return np.clip(raw.real, -cap, cap) + 1j * np.clip(raw.imag, -cap, cap)


def _parts(sys, phi):
    G = afqmc.green(sys, phi)
    e1 = sum(np.einsum("ij,wji->w", sys.h1, Gs) for Gs in G)
    rb = afqmc.rhobar(sys, G)
    return e1, 0.5 * np.sum(rb * rb, axis=1)


def _eloc_no_half(sys, phi, chunk=0):
    e = ORIG["local_energy"](sys, phi, chunk)
    e1, _ = _parts(sys, phi)
    return e1 + 2 * (e - e1)


def _eloc_no_exchange(sys, phi, chunk=0):
    e1, coul = _parts(sys, phi)
    return e1 + coul


def _eloc_exchange_sign(sys, phi, chunk=0):
    e = ORIG["local_energy"](sys, phi, chunk)
    e1, coul = _parts(sys, phi)
    return e1 + coul + (e1 + coul - e)


def _step_variant(kind):
    def step(sys, phi, logO, x, xbar):
        phi3, logO3, logR, logI = ORIG["step_determinant"](sys, phi, logO, x, xbar)
        if kind == "conjugated xbar^2":
            logI = logI + 0.5 * np.sum(xbar * xbar, axis=1) - 0.5 * np.sum(np.abs(xbar) ** 2, axis=1)
        elif kind == "x.xbar sign":
            logI = logI - 2 * np.sum(x * xbar, axis=1)
        elif kind == "mean-field scalar dropped":
            log_s = -1j * sys.sqrt_dt * ((x - xbar) @ sys.rho_mf)
            logR, logI = logR - log_s, logI - log_s
        elif kind == "energy shift sign":
            logI = logI + 2 * sys.dt * (sys.C - sys.E_T)
        return phi3, logO3, logR, logI
    return step


def _propagate_no_cos(sys, wk, x):
    """The phaseless update without the max(0, cos dtheta) factor."""
    if sys.mode != afqmc.PHASELESS:
        return ORIG["propagate"](sys, wk, x)
    live = wk.alive
    if not np.any(live):
        return
    phi = wk.phi[live]
    xs = np.asarray(x, dtype=np.float64)[live]
    xbar = afqmc.force_bias(sys, afqmc.green(sys, phi))
    phi3, logO_new, logR, logI = afqmc.step_determinant(sys, phi, wk.logO[live], xs, xbar)
    idx = np.nonzero(live)[0]
    wk.phi[idx] = phi3
    wk.logO[idx] = logO_new
    wk.w[idx] = (wk.w[live].real * np.exp(logI.real)).astype(np.complex128)


def _comb_left(w, n_out, u):
    """The comb taking the first walker whose running sum reaches the point (side='left'):
    a dead walker sitting on a boundary can be chosen."""
    w = np.asarray(w, dtype=np.float64)
    W = float(w.sum())
    points = (np.arange(n_out) + float(u)) * (W / n_out)
    return np.minimum(np.searchsorted(np.cumsum(w), points, side="left"), w.size - 1), W / n_out


def _seed_variant(kind):
    def seed(sA, sB, wkA):
        if kind == "inverted ratio":
            phi = wkA.phi[:, :, pes.seed_columns(sA, sB)]
            logR = wkA.logO - afqmc.overlap(sB, phi)
            w = wkA.w.real * np.exp(logR.real) * np.maximum(0.0, np.cos(logR.imag))
            return afqmc.Walkers(sB, phi.shape[0], phi=phi, w=np.where(wkA.alive, w, 0.0) + 0j)
        wkB = ORIG_PES["seed_secondary"](sA, sB, wkA)
        if kind == "phase not projected":
            phi = wkB.phi
            logR = afqmc.overlap(sB, phi) - wkA.logO
            w = wkA.w.real * np.exp(logR.real)
            return afqmc.Walkers(sB, phi.shape[0], phi=phi, w=w + 0j)
        return wkB
    return seed


def _last_columns(sA, sB):
    return (list(range(sA.n_up - sB.n_up, sA.n_up)) +
            list(range(sA.N - sB.n_dn, sA.N)))


def _per_tau_ddof0(dE):
    dE = np.asarray(dE, dtype=np.float64)
    return dE.mean(axis=1), dE.std(axis=1, ddof=0) / np.sqrt(dE.shape[1])


def _cumulative_strict(dE, taus, tau_eq):
    return ORIG_STATS["cumulative"](dE, taus, np.nextafter(tau_eq, np.inf))


def _estimate_latest_minimum(dE, taus, tau_eq):
    t, C = stats.cumulative(dE, taus, tau_eq)
    mean, se = stats.per_tau(C)
    i = len(se) - 1 - int(np.nanargmin(se[::-1]))
    return float(mean[i]), float(se[i]), float(t[i])


def _ortho_stale_logO(sys, wk):
    saved = wk.logO.copy()
    ORIG["orthonormalise"](sys, wk)
    wk.logO[:] = saved


MUTANTS = {
    "force bias sign": ("force_bias", lambda s, G: -ORIG["force_bias"](s, G)),
    "force bias without <rho>_T": ("force_bias", _fb_no_mean_field),
    "force bias without i": ("force_bias", lambda s, G: -1j * ORIG["force_bias"](s, G)),
    "cap per component": ("force_bias", _fb_cap_componentwise),
    "G transposed": ("green", lambda s, phi: [np.swapaxes(g, 1, 2) for g in ORIG["green"](s, phi)]),
    "overlap of conj(Phi)": ("overlap", lambda s, phi: ORIG["overlap"](s, np.conj(phi))),
    "E_L without 1/2": ("local_energy", _eloc_no_half),
    "E_L without exchange": ("local_energy", _eloc_no_exchange),
    "E_L exchange sign": ("local_energy", _eloc_exchange_sign),
    "Taylor one order short": ("taylor_apply", lambda A, phi, n: ORIG["taylor_apply"](A, phi, n - 1)),
    "xbar^2 conjugated": ("step_determinant", _step_variant("conjugated xbar^2")),
    "x.xbar sign": ("step_determinant", _step_variant("x.xbar sign")),
    "mean-field scalar dropped": ("step_determinant", _step_variant("mean-field scalar dropped")),
    "energy shift sign": ("step_determinant", _step_variant("energy shift sign")),
    "phaseless cos factor dropped": ("propagate", _propagate_no_cos),
    "log O stale after MGS": ("orthonormalise", _ortho_stale_logO),
    "MGS not normalised": ("modified_gram_schmidt", lambda q: 2.0 * ORIG["modified_gram_schmidt"](q)),
    "K without -1/2 sum L L": ("__init__", _reinit(_k_without_LL)),
    "K mean-field sign": ("__init__", _reinit(_k_mean_field_sign)),
    "C sign": ("__init__", _reinit(lambda s: setattr(s, "C", -s.C))),
    "full one-body step on each side": ("__init__", _reinit(_full_step)),
    "comb picks on the left of a point": ("pes.comb_select", _comb_left),
    "seeding ratio inverted": ("pes.seed_secondary", _seed_variant("inverted ratio")),
    "seeding phase not projected": ("pes.seed_secondary", _seed_variant("phase not projected")),
    "seeding keeps the last columns": ("pes.seed_columns", _last_columns),
    "standard error with ddof 0": ("stats.per_tau", _per_tau_ddof0),
    "equilibration cut tau > tau_eq": ("stats.cumulative", _cumulative_strict),
    "latest instead of earliest minimum": ("stats.delta_e_estimate", _estimate_latest_minimum),
    "Box-Muller radius without 2": ("box_muller",
                                    lambda u1, u2: tuple(z / np.sqrt(2) for z in ORIG_BOX_MULLER(u1, u2))),
}


def first_failing_pin():
    for name, pin in PINS:
        try:
            pin()
        except Exception:   # an assertion, or a pin that cannot even run on the mutant
            return name
    return None


def test_control_passes_every_pin():
    assert first_failing_pin() is None


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(monkeypatch, mutant):
    target, fn = MUTANTS[mutant]
    if target == "__init__":
        monkeypatch.setattr(afqmc.System, "__init__", fn)
    elif target == "box_muller":
        monkeypatch.setattr(philox, "box_muller", fn)
    elif target.startswith("pes."):
        monkeypatch.setattr(pes, target[4:], fn)
    elif target.startswith("stats."):
        monkeypatch.setattr(stats, target[6:], fn)
    else:
        monkeypatch.setattr(afqmc, target, fn)
    assert first_failing_pin() is not None, f"no pin catches: {mutant}"
