"""Split-precision path (AFQMC_BF16X3) against the FP64 oracle and the FP64 GPU path.

Both paths take the same fields, so their difference is deterministic.  Criteria:
per-walker weights and local energies within the accumulated error of the split
arithmetic (the tensor-core products carry ~2^-16 relative error, propagated through
50 steps), and, the method's target, the correlated-pair energy difference within
0.1 mHa of the FP64 path.  The measured errors are written as JSON to the directory named
by AFQMC_REPORT_DIR, when set.
"""
import json
import os

import numpy as np
import pytest

from gpu_util import need_gpu, system_data
from oracle import afqmc as orc
from synthetic import CONFIGS, explicit_fields

pytestmark = pytest.mark.gpu
OUT = os.environ.get("AFQMC_REPORT_DIR", "")
REPORT = {}


def dump():
    if OUT and os.path.isdir(OUT):
        with open(os.path.join(OUT, "mixed_errors.json"), "w") as f:
            json.dump(REPORT, f, indent=1)


def gpu_sys(afq, d, nw, dt, precision, seed=1, R=1):
    return afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=dt, n_walkers=nw,
                      seed=seed, n_repeats=R, precision=precision)


# (select_kernel) propagation: 4 tensor cores (streamed V_HS, M <= 256), 3 tensor cores (M <= 64),
# 2 fused FP32 kernel, 1 FP32 GEMMs + Taylor kernel; local energy: 0 tensor cores, 2 / 4 / 8
# FP32 kernel with that many walkers per CTA
@pytest.mark.parametrize("cfg,which,coupling,nw,taylor,energy,mgs", [
    ("C1", "A", 1.0, 128, 3, 0, 0), ("C1", "A", 1.0, 128, 2, 4, 1), ("C1", "B", 1.0, 128, 3, 0, 1),
    ("C1", "B", 1.0, 128, 4, 0, 0), ("C2", "B", "moderate", 96, 3, 0, 0),
    ("C2", "B", "moderate", 96, 2, 0, 1), ("C2", "A", "moderate", 96, 1, 8, 0),
    ("C2", "A", "moderate", 96, 4, 0, 1)])
def test_mixed_walkers_track_fp64_oracle(cfg, which, coupling, nw, taylor, energy, mgs):
    """Each kernel variant, forced, against the oracle after 50 steps on the same fields.  Bars:
    1e-4 relative on E_L, 1e-3 on w, 1e-4 Ha on the mixed energy, about ten times the errors
    measured at these shapes (E_L ~1e-5, w ~1e-4, mixed energy ~1e-5 Ha)."""
    afq = need_gpu()
    d = system_data(cfg, which, coupling)
    dt = CONFIGS[cfg]["dt"]
    fields = explicit_fields(50, nw, d["X"], seed=8)
    g = gpu_sys(afq, d, nw, dt, afq.BF16X3)
    g.select_kernel(afq.K_TAYLOR, taylor)
    g.select_kernel(afq.K_EXCHANGE, energy)
    g.select_kernel(afq.K_MGS, mgs)
    info = g.info()
    assert (info.tuned_taylor_smem, info.tuned_energy_walkers_per_cta,
            info.tuned_orthonormalise) == (taylor, energy, mgs)
    o = orc.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt)
    wk = orc.Walkers(o, nw)
    errs = []
    for blk in range(10):
        g.propagate(5, fields[5 * blk:5 * blk + 5])
        for t in range(5 * blk, 5 * blk + 5):
            orc.propagate(o, wk, fields[t])
        g.orthonormalise()
        orc.orthonormalise(o, wk)
    el, em, _ = g.energy()
    el_o = orc.local_energy(o, wk.phi)
    st = g.state()
    live = wk.alive & st["alive"]
    assert live.sum() >= 0.9 * wk.alive.sum()
    e_rel = np.max(np.abs(el[live] - el_o[live]) / np.abs(el_o[live]))
    w_rel = np.max(np.abs(st["w"].real[live] - wk.w.real[live]) / np.abs(wk.w.real[live]))
    em_o, _ = orc.mixed_energy(o, wk.w, el_o, np.zeros(nw, int), 1)
    REPORT[f"{cfg}{which}_taylor{taylor}_energy{energy}_mgs{mgs}"] = dict(
        max_rel_E_L=float(e_rel), max_rel_w=float(w_rel), mixed_E_err_Ha=float(em[0] - em_o[0]))
    dump()
    assert e_rel < 1e-4 and w_rel < 1e-3, (e_rel, w_rel)
    assert abs(em[0] - em_o[0]) < 1e-4


def test_mixed_pair_delta_E_within_0p1_mHa_of_fp64():
    """C2 at full size, moderate coupling: the correlated pair in both precisions, same fields."""
    afq = need_gpu()
    cfg = CONFIGS["C2"]
    nw, R, steps = cfg["n_walkers"], 11, 200
    dA, dB = system_data("C2", "A", "moderate"), system_data("C2", "B", "moderate")
    res = {}
    for prec in (afq.FP64, afq.BF16X3):
        A = gpu_sys(afq, dA, nw, cfg["dt"], prec, R=R)
        B = gpu_sys(afq, dB, nw, cfg["dt"], prec, R=R)
        res[prec] = afq.pair_delta_E(A, B, steps, 5, 5, tau_eq=0.25)
        A.close()
        B.close()
    f, m = res[afq.FP64], res[afq.BF16X3]
    dE_f = f["E"][:, 1, :] - f["E"][:, 0, :]
    dE_m = m["E"][:, 1, :] - m["E"][:, 0, :]
    err_series = np.abs(dE_m - dE_f).max()
    err_E = np.abs(m["E"] - f["E"]).max()
    REPORT["C2_pair"] = dict(max_abs_dE_err_mHa=1e3 * float(err_series),
                             max_abs_E_err_mHa=1e3 * float(err_E),
                             estimate_fp64=[f["dE_mean"], f["dE_sigma"]],
                             estimate_bf16x3=[m["dE_mean"], m["dE_sigma"]],
                             estimate_diff_mHa=1e3 * abs(m["dE_mean"] - f["dE_mean"]))
    dump()
    # the estimate (cumulative averages after tau_eq, 11 repeats) within 0.1 mHa, same error bar
    assert abs(m["dE_mean"] - f["dE_mean"]) < 1e-4
    assert abs(m["dE_sigma"] / f["dE_sigma"] - 1) < 0.05
    # per-tau means over the repeats stay close (single-repeat values drift further apart)
    assert np.abs(dE_m.mean(axis=1) - dE_f.mean(axis=1)).max() < 5e-4


def test_autotuner_picks_valid_variants_and_persists(tmp_path):
    afq = need_gpu()
    d = system_data("C2", "A", "moderate")
    cache = tmp_path / "tune.json"
    s1 = gpu_sys(afq, d, 512, 0.005, afq.BF16X3)
    s1.close()
    s2 = afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=0.005, n_walkers=512,
                    precision=afq.BF16X3, autotune_cache=str(cache))
    info = s2.info()
    assert info.tuned_energy_walkers_per_cta in (0, 2, 4, 8)
    assert info.tuned_taylor_smem in (0, 1, 2, 3, 4)
    text = cache.read_text()
    assert "energy_v2:M64X320u8d8w512" in text and "propagate_v3" in text
    s2.close()
    # a second setup of the same shape reads the choices back
    s3 = afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=0.005, n_walkers=512,
                    precision=afq.BF16X3, autotune_cache=str(cache))
    i3 = s3.info()
    assert (i3.tuned_energy_walkers_per_cta, i3.tuned_taylor_smem) == \
        (info.tuned_energy_walkers_per_cta, info.tuned_taylor_smem)
    s3.close()
    s4 = afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=0.005, n_walkers=512,
                    precision=afq.FP64)
    assert s4.info().tuned_energy_walkers_per_cta == -1
    s4.close()


@pytest.mark.parametrize("cfg,which", [("C2", "B"), ("C3", "B")])
def test_cholesky_qr_orthonormalises_and_lowers_log_overlap(cfg, which):
    """Cholesky QR (K_MGS 1): per spin block Q^H Q = I (Q in FP32), Q spans the walker's
    columns (the energy, invariant under Phi -> Phi R^{-1}, is unchanged), log O lowered by
    log det R agrees with a recomputation, and Q equals the oracle's modified Gram-Schmidt."""
    afq = need_gpu()
    d = system_data(cfg, which, "moderate")
    nw = 64
    g = gpu_sys(afq, d, nw, CONFIGS[cfg]["dt"], afq.BF16X3)
    g.select_kernel(afq.K_MGS, 1)
    g.propagate(5, explicit_fields(5, nw, d["X"], seed=23))
    before = g.state()
    _, em0, _ = g.energy()
    g.orthonormalise()
    after = g.state()
    _, em1, _ = g.energy()
    o = orc.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], CONFIGS[cfg]["dt"])
    for a, b in o.spins:
        Q = after["phi"][:, :, a:b]
        gram = np.einsum("wia,wib->wab", Q.conj(), Q)
        assert np.abs(gram - np.eye(b - a)).max() < 5e-6
        ref = orc.modified_gram_schmidt(before["phi"][:, :, a:b])
        assert np.abs(Q - ref).max() < 5e-6
    assert abs(em1[0] - em0[0]) < 1e-5 * abs(em0[0])
    live = before["alive"]
    rec = orc.overlap(o, after["phi"])
    assert np.abs(np.exp(after["logO"][live] - rec[live]) - 1).max() < 1e-5
    g.close()


# The split path's overlap update sums Psi^T Phi' in FP32, so its log O carries ~1e-6 of
# rounding against an FP64 recomputation.  That error does not accumulate in the weights: each
# step's ratio log O(Phi') - log O(Phi) cancels the previous step's error (the sum telescopes),
# so a weight carries at most the last update's rounding.
LOGO_F32 = 1e-5


def test_gram_schmidt_log_overlap_update_matches_recomputation():
    """Split path: Gram-Schmidt lowers log O by sum_j log R_jj (Sec. II.D; Phi -> Phi R^{-1}) instead
    of recomputing the overlaps.  A refresh (the timing call's refresh form recomputes log O and
    Theta from the walkers in FP64) must land on the same values, up to the FP32 rounding of the
    overlap update."""
    afq = need_gpu()
    d = system_data("C2", "B", "moderate")
    nw = 64
    g = gpu_sys(afq, d, nw, CONFIGS["C2"]["dt"], afq.BF16X3)
    g.propagate(5, explicit_fields(5, nw, d["X"], seed=21))
    g.orthonormalise()
    before = g.state()
    _, em0, _ = g.energy()
    afq.afqmc_time_kernel(g.h, afq.K_OVERLAP, 1)
    after = g.state()
    _, em1, _ = g.energy()
    g.close()
    live = before["alive"]
    assert live.sum() >= nw - 2
    assert np.abs(after["logO"].real - before["logO"].real)[live].max() < LOGO_F32
    dphase = np.angle(np.exp(1j * (after["logO"].imag - before["logO"].imag)))
    assert np.abs(dphase[live]).max() < LOGO_F32
    assert abs(em1[0] - em0[0]) < 1e-5 * abs(em0[0])


def test_kernel_timing_leaves_the_walkers_unchanged():
    afq = need_gpu()
    d = system_data("C2", "B", "moderate")
    nw = 64
    g = gpu_sys(afq, d, nw, CONFIGS["C2"]["dt"], afq.BF16X3)
    g.propagate(5, explicit_fields(5, nw, d["X"], seed=22))
    g.orthonormalise()
    before = g.state()
    _, em0, _ = g.energy()
    for k in (afq.K_VHS, afq.K_FORCE_BIAS, afq.K_TAYLOR, afq.K_EXCHANGE, afq.K_OVERLAP,
              afq.K_OVERLAP_UPDATE):
        assert afq.afqmc_time_kernel(g.h, k, 2) > 0
    after = g.state()
    _, em1, _ = g.energy()
    assert np.array_equal(after["phi"], before["phi"])
    assert np.array_equal(after["w"], before["w"])
    assert np.array_equal(after["alive"], before["alive"])
    live = before["alive"]
    assert np.abs(after["logO"].real - before["logO"].real)[live].max() < LOGO_F32
    assert abs(em1[0] - em0[0]) < 1e-5 * abs(em0[0])
    # Gram-Schmidt of walkers that are already orthonormal changes them only by rounding
    assert afq.afqmc_time_kernel(g.h, afq.K_MGS, 2) > 0
    again = g.state()
    assert np.abs(again["phi"] - before["phi"]).max() < 1e-5 * np.abs(before["phi"]).max()
    assert np.abs(again["logO"].real - before["logO"].real)[live].max() < 1e-5
    assert np.array_equal(again["w"], before["w"])
    g.close()
    f = gpu_sys(afq, d, 8, CONFIGS["C2"]["dt"], afq.FP64)
    with pytest.raises(RuntimeError):
        afq.afqmc_time_kernel(f.h, afq.K_OVERLAP_UPDATE, 1)
    assert afq.afqmc_time_kernel(f.h, afq.K_MGS, 2) > 0
    f.close()
