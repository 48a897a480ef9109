"""Tensor-core local energy of the split-precision step (split-BF16 tcgen05 GEMM of
Psi^T L_g Theta with the exchange / Coulomb reduction in the TMEM epilogue).

On the same walkers the split-precision handle's E_L, with the tensor-core kernel and with
the FP32 kernel forced, is compared walker by walker with the FP64 handle's E_L.  A split
BF16 product carries ~2^-16 relative error (the dropped lo*lo term), so the two-body energy
of a walker differs from FP64 by ~1e-5 to 1e-4 Ha at C2 (a CPU emulation of the same
arithmetic on the same walkers gives the same per-walker differences), and the mean over
walkers by ~1e-5 Ha; the FP32 kernel is ~10x closer.  Walkers are the trial plus complex
noise, orthonormalised per spin as the propagation keeps them.  Shapes cover every orbital
padding (8, 16, 32 rows per Cholesky vector), one to four 64-wide k slices (M = 64 to 200; above
64 one product per spin block, 4 to 16 rows per Cholesky vector and spin), spin-unbalanced
blocks and walker counts that leave a ragged last tile.  The measured errors
are written as JSON to the directory named by AFQMC_REPORT_DIR, when set.

Per-walker bounds grow with the condition number kappa of the walker's overlap matrices
Psi_s^T Phi_s (the larger of the two spins): Theta = Phi O^-1 passes the relative rounding
errors of its operands on amplified by up to kappa, and the noisy test walkers reach kappa ~ 500
at M = 128.  A CPU emulation of the split products (hi*hi + hi*lo + lo*hi of the rounded
operands, exact sums) on the C3 walkers gives |dE| <= 7e-6 kappa Ha; the bound below is
2e-4 + 3e-5 kappa (FP32 kernel: 1e-4 + 3e-6 kappa).  Mean and bias over the walkers keep
fixed bounds.
"""
import json
import os

import numpy as np
import pytest

from gpu_util import need_gpu, system_data
from synthetic import build_system

pytestmark = pytest.mark.gpu
OUT = os.environ.get("AFQMC_REPORT_DIR", "")
REPORT = {}


def walkers(d, nw, seed, scale=0.2):
    rng = np.random.default_rng(seed)
    psi = d["trial"]
    phi = psi[None].astype(complex) + scale * (rng.standard_normal((nw,) + psi.shape) +
                                               1j * rng.standard_normal((nw,) + psi.shape))
    nu = d["n_up"]
    for a, b in ((0, nu), (nu, psi.shape[1])):
        if b > a:
            phi[:, :, a:b] = np.linalg.qr(phi[:, :, a:b])[0]
    return phi


def overlap_kappa(d, phi):
    """Condition number of Psi_s^T Phi_s per walker, the larger of the two spins."""
    psi, nu = d["trial"], d["n_up"]
    out = np.ones(phi.shape[0])
    for a, b in ((0, nu), (nu, psi.shape[1])):
        if b > a:
            out = np.maximum(out, np.linalg.cond(np.einsum("mi,wmj->wij", psi[:, a:b], phi[:, :, a:b])))
    return out


def energies(afq, d, phi, precision, variant=None):
    nw = phi.shape[0]
    s = afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=0.005, n_walkers=nw,
                   precision=precision, autotune=False)
    if variant is not None:
        s.select_kernel(afq.K_EXCHANGE, variant)
    s.set_walkers(phi)
    el, _, _ = s.energy()
    el2, _, _ = s.energy()
    s.close()
    return el, el2


SMALL_SPIN = dict(M=80, X=160, n_up=3, n_dn=2, seed=1703, coupling="moderate")   # 4 rows per g and spin, M > 64


@pytest.mark.parametrize("cfg,which,coupling,nw", [
    ("C1", "A", 1.0, 37),            # 2/2: 8 padded rows per g, 16 walkers per tile
    ("C1", "B", 1.0, 5),             # 2/1, fewer walkers than one tile
    ("C2", "A", "moderate", 300),    # 8/8: 16 rows per g
    ("C2", "B", "moderate", 129),    # 8/7
    # M > 64: one product per spin block (P2 = 4, 8, 16 rows per g and spin)
    ("C5", "A", "moderate", 70),     # 12/12, M = 96 -> two k slices
    ("C3", "A", "moderate", 300),    # 16/16, M = 128
    ("C3", "B", "moderate", 257),    # 16/15
    ("C4", "A", "moderate", 100),    # 9/9, M = 200 -> four k slices, ragged
    ("C4", "B", "moderate", 90),     # 8/8, M = 190
    ("small", None, 1.0, 65),        # 3/2, M = 80
])
def test_tensor_core_energy_matches_fp64(cfg, which, coupling, nw):
    afq = need_gpu()
    d = build_system(**SMALL_SPIN) if cfg == "small" else system_data(cfg, which, coupling)
    phi = walkers(d, nw, seed=11)
    e64, _ = energies(afq, d, phi, afq.FP64)
    etc, etc2 = energies(afq, d, phi, afq.BF16X3, variant=0)
    e32, _ = energies(afq, d, phi, afq.BF16X3, variant=2)
    d_tc, d_32 = np.abs(etc - e64), np.abs(e32 - e64)
    REPORT[f"{cfg}{which or ''}"] = dict(tc_max_Ha=float(d_tc.max()), tc_mean_Ha=float(d_tc.mean()),
                                   tc_bias_Ha=float(np.mean(etc.real - e64.real)),
                                   f32_max_Ha=float(d_32.max()), f32_mean_Ha=float(d_32.mean()))
    if OUT and os.path.isdir(OUT):
        with open(os.path.join(OUT, "energy_tc_errors.json"), "w") as f:
            json.dump(REPORT, f, indent=1)
    kap = overlap_kappa(d, phi)
    REPORT[f"{cfg}{which or ''}"].update(kappa_max=float(kap.max()),
                                         tc_max_over_kappa=float(np.max(d_tc / kap)))
    if OUT and os.path.isdir(OUT):
        with open(os.path.join(OUT, "energy_tc_errors.json"), "w") as f:
            json.dump(REPORT, f, indent=1)
    assert np.array_equal(etc, etc2)                     # fixed-order sums: reproducible
    assert np.all(d_32 <= 1e-4 + 3e-6 * kap)
    assert np.all(d_tc <= 2e-4 + 3e-5 * kap) and d_tc.mean() < 2e-4
    assert abs(np.mean(etc.real - e64.real)) < 5e-5


def test_select_kernel_rejects_unsupported_variants():
    afq = need_gpu()
    d = system_data("C1", "A")
    s = afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=0.01, n_walkers=8,
                   precision=afq.BF16X3, autotune=False)
    with pytest.raises(RuntimeError):
        s.select_kernel(afq.K_EXCHANGE, 3)
    with pytest.raises(RuntimeError):
        s.select_kernel(afq.K_VHS, 0)
    s.select_kernel(afq.K_EXCHANGE, 4)
    assert s.info().tuned_energy_walkers_per_cta == 4
    s.close()
    f = afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=0.01, n_walkers=8)
    with pytest.raises(RuntimeError):
        f.select_kernel(afq.K_EXCHANGE, 0)
    f.close()
