"""Long runs: the GPU path and the oracle on independent field streams agree statistically.

C1 pair (M = 8, Nchol = 24, 2/2 vs 2/1), 256 walkers, 600 steps of dt = 0.01 (tau = 6 Ha^-1),
energy and Gram-Schmidt every 5 steps.  Without population control the weights degenerate as
tau grows, so a run's late energies are dominated by few walkers and the error bar from the
spread of its repeat groups understates the run-to-run scatter (measured on the oracle over 14
seeds: standard deviation 7.2 mHa for the ion against a typical within-run error of 4.8 mHa).
The comparison therefore takes its sigma from independent runs: the GPU on 16 seeds, the
oracle on 8 other seeds (with only 4 the oracle's own spread is too uncertain to serve as an
error bar); for each run the mixed energies of both systems (Eq. 7, Eq. 10) are
averaged over tau >= 1, and the seed means of E_A, E_B and the correlated difference
Delta E = E_B - E_A (Sec. II.B) must agree within two combined standard errors.  Both
precisions are held to it.  Seeds are fixed, so the outcome is deterministic.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, system_data
from oracle import afqmc as orc
from synthetic import CONFIGS

pytestmark = pytest.mark.gpu

NW, R, STEPS, TAU_EQ = 256, 8, 600, 1.0
GPU_SEEDS = list(range(1, 17))
ORACLE_SEEDS = [202, 303, 404, 505, 606, 707, 808, 909]


def run_means(EA, EB, taus):
    """(E_A, E_B, Delta E) of one run: time averages over tau >= TAU_EQ, all repeat groups"""
    sel = taus >= TAU_EQ
    a, b = EA[sel].mean(), EB[sel].mean()
    return np.array([a, b, b - a])


@pytest.fixture(scope="module")
def oracle_runs():
    dt = CONFIGS["C1"]["dt"]
    dA, dB = system_data("C1", "A"), system_data("C1", "B")
    oA = orc.System(dA["h1"], dA["L"], dA["trial"], dA["n_up"], dA["n_dn"], dt)
    oB = orc.System(dB["h1"], dB["L"], dB["trial"], dB["n_up"], dB["n_dn"], dt)
    out = []
    for seed in ORACLE_SEEDS:
        ref = orc.run_pair(oA, oB, NW, STEPS, seed=seed, n_repeats=R)
        taus = np.asarray(ref["steps"]) * dt
        out.append(run_means(np.asarray(ref["E"][0]), np.asarray(ref["E"][1]), taus))
    return np.array(out)


@pytest.mark.parametrize("precision", ["FP64", "BF16X3"])
def test_long_runs_agree_with_oracle_within_two_sigma(oracle_runs, precision):
    afq = need_gpu()
    dt = CONFIGS["C1"]["dt"]
    dA, dB = system_data("C1", "A"), system_data("C1", "B")
    prec = getattr(afq, precision)
    got = []
    for seed in GPU_SEEDS:
        gA = afq.System(dA["h1"], dA["L"], dA["trial"], dA["n_up"], dA["n_dn"], dt=dt,
                        n_walkers=NW, seed=seed, n_repeats=R, precision=prec)
        gB = afq.System(dB["h1"], dB["L"], dB["trial"], dB["n_up"], dB["n_dn"], dt=dt,
                        n_walkers=NW, seed=seed, n_repeats=R, precision=prec)
        res = afq.pair_delta_E(gA, gB, STEPS, energy_every=5, mgs_every=5, tau_eq=TAU_EQ)
        gA.close()
        gB.close()
        got.append(run_means(res["E"][:, 0, :], res["E"][:, 1, :], res["taus"]))
    got = np.array(got)
    g, gs = got.mean(axis=0), got.std(axis=0, ddof=1) / np.sqrt(len(got))
    o, os_ = oracle_runs.mean(axis=0), oracle_runs.std(axis=0, ddof=1) / np.sqrt(len(oracle_runs))
    for q, name in enumerate(("E_A", "E_B", "dE")):
        assert np.isfinite(g[q]) and gs[q] > 0 and os_[q] > 0
        assert abs(g[q] - o[q]) < 2.0 * np.hypot(gs[q], os_[q]), (name, g[q], gs[q], o[q], os_[q])


def test_c2_long_run_split_matches_fp64():
    """C2 pair (M = 64, Nchol = 320, 8/8 vs 8/7, 2048 walkers, 11 repeats) over 2000 steps of
    dt = 0.005 (tau = 10 Ha^-1), moderate coupling: the split-precision path against the FP64
    path on the same field stream.  The FP64 path is held to the oracle walker by walker at
    1e-9, so this carries that agreement to a long run: the correlated Delta E (cumulative
    averages after tau_eq = 2.5) of the two paths within 0.1 mHa and within the FP64 run's
    standard error."""
    afq = need_gpu()
    dA, dB = system_data("C2", "A", "moderate"), system_data("C2", "B", "moderate")
    dt, nw, R, steps = CONFIGS["C2"]["dt"], 2048, 11, 2000
    out = {}
    for precision in ("FP64", "BF16X3"):
        hs = [afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=dt, n_walkers=nw,
                         seed=1, n_repeats=R, precision=getattr(afq, precision))
              for d in (dA, dB)]
        out[precision] = afq.pair_delta_E(hs[0], hs[1], steps, energy_every=5, mgs_every=5,
                                          tau_eq=2.5)
        for h in hs:
            h.close()
    d = abs(out["BF16X3"]["dE_mean"] - out["FP64"]["dE_mean"])
    sigma = out["FP64"]["dE_sigma"]
    assert np.isfinite(d) and sigma > 0
    assert d < 1e-4 and d < sigma, (out["BF16X3"]["dE_mean"], out["FP64"]["dE_mean"], sigma)
