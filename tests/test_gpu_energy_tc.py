"""Tensor-core local energy of the split-precision step (split-BF16 tcgen05 GEMM of
Psi^T L_g Theta with the exchange / Coulomb reduction in the TMEM epilogue).

On the same walkers the split-precision handle's E_L, with the tensor-core kernel and with
the FP32 kernel forced, is compared walker by walker with the FP64 handle's E_L.  A split
BF16 product carries ~2^-16 relative error (the dropped lo*lo term), so the two-body energy
of a walker differs from FP64 by ~1e-5 to 1e-4 Ha at C2 (a CPU emulation of the same
arithmetic on the same walkers gives the same per-walker differences), and the mean over
walkers by ~1e-5 Ha; the FP32 kernel is ~10x closer.  Walkers are the trial plus complex
noise, orthonormalised per spin as the propagation keeps them.  Shapes cover every orbital
padding (8, 16, 32 rows per Cholesky vector), one and two 64-wide k slices (M = 64, 96),
spin-unbalanced blocks and walker counts that leave a ragged last tile.  The measured errors
are written as JSON to the directory named by AFQMC_REPORT_DIR, when set.
"""
import json
import os

import numpy as np
import pytest

from gpu_util import need_gpu, system_data

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


@pytest.mark.parametrize("cfg,which,coupling,nw", [
    ("C1", "A", 1.0, 37),            # 2/2: 8 padded rows per g, 16 walkers per tile
    ("C1", "B", 1.0, 5),             # 2/1, fewer walkers than one tile
    ("C2", "A", "moderate", 300),    # 8/8: 16 rows per g
    ("C2", "B", "moderate", 129),    # 8/7
    ("C5", "A", "moderate", 70),     # 12/12: 32 rows per g, M = 96 -> two k slices
])
def test_tensor_core_energy_matches_fp64(cfg, which, coupling, nw):
    afq = need_gpu()
    d = system_data(cfg, which, coupling)
    phi = walkers(d, nw, seed=11)
    e64, _ = energies(afq, d, phi, afq.FP64)
    etc, etc2 = energies(afq, d, phi, afq.BF16X3, variant=0)
    e32, _ = energies(afq, d, phi, afq.BF16X3, variant=2)
    d_tc, d_32 = np.abs(etc - e64), np.abs(e32 - e64)
    REPORT[f"{cfg}{which}"] = dict(tc_max_Ha=float(d_tc.max()), tc_mean_Ha=float(d_tc.mean()),
                                   tc_bias_Ha=float(np.mean(etc.real - e64.real)),
                                   f32_max_Ha=float(d_32.max()), f32_mean_Ha=float(d_32.mean()))
    if OUT and os.path.isdir(OUT):
        with open(os.path.join(OUT, "energy_tc_errors.json"), "w") as f:
            json.dump(REPORT, f, indent=1)
    assert np.array_equal(etc, etc2)                     # fixed-order sums: reproducible
    assert d_32.max() < 2e-4
    assert d_tc.max() < 2e-3 and d_tc.mean() < 2e-4
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
