"""CPU emulation of the split-BF16 two-body local energy (Eq. 10 through T_g = L~_g Theta,
Sec. II.D) at the C3 shape, against the per-walker bound the GPU test of the tensor-core energy
uses (`test_tensor_core_energy_matches_fp64`: |dE| <= 2e-4 + 3e-5 kappa Ha, kappa the larger
condition number of the walker's overlap matrices Psi_s^T Phi_s).

The kernel holds L~_g = Psi_s^T L_g (from FP64) and Theta_s (from the FP32 overlap kernel) as
x = hi + lo with hi = bf16(x), lo = bf16(x - hi), and forms every T_g from the three products
hi*hi + hi*lo + lo*hi.  The emulation rounds the operands the same way (round to nearest even
to bfloat16, written out here from the format's definition) and sums the three products
exactly, so it measures the error of the split itself; the kernel's FP32 accumulation adds
~2^-24 relative on top.  Theta's own FP32 rounding passes through O^-1, which is why the bound
grows with kappa.  The restatement of E_L through T_g is first pinned to the oracle's E_L in
FP64.
"""
import numpy as np
import pytest

from oracle import afqmc as orc
from synthetic import CONFIGS, build_system

BOUND = (2e-4, 3e-5)   # the GPU test's per-walker bound: BOUND[0] + BOUND[1] * kappa (Ha)


def bf16(x):
    """float32 -> nearest bfloat16 (ties to even), returned as float32."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    r = (b + np.uint32(0x7FFF) + ((b >> np.uint32(16)) & np.uint32(1))) & np.uint32(0xFFFF0000)
    return r.view(np.float32)


def split(x64):
    """hi = bf16(fp32(x)), lo = bf16(fp32(x - hi)), both as float64."""
    hi = bf16(np.asarray(x64, dtype=np.float32)).astype(np.float64)
    lo = bf16((np.asarray(x64, dtype=np.float64) - hi).astype(np.float32)).astype(np.float64)
    return hi, lo


def walkers(d, nw, seed, scale=0.2):
    """The trial plus complex noise, each spin block orthonormalised."""
    rng = np.random.default_rng(seed)
    psi = d["trial"]
    phi = psi[None].astype(complex) + scale * (rng.standard_normal((nw,) + psi.shape) +
                                               1j * rng.standard_normal((nw,) + psi.shape))
    for a, b in ((0, d["n_up"]), (d["n_up"], psi.shape[1])):
        if b > a:
            phi[:, :, a:b] = np.linalg.qr(phi[:, :, a:b])[0]
    return phi


def energy_terms(d, phi, products):
    """One-body part and two-body part of E_L per walker; `products(Lt, Th)` forms
    T[w, g, a, b] = sum_i Lt[g, a, i] Th[w, i, b] (Lt real, Th complex)."""
    psi, L, h1 = d["trial"], d["L"], d["h1"]
    spins = [(0, d["n_up"]), (d["n_up"], psi.shape[1])]
    e1 = np.zeros(phi.shape[0], complex)
    tr = 0
    ex = np.zeros(phi.shape[0], complex)
    kappa = np.ones(phi.shape[0])
    for a, b in spins:
        ps, ph = psi[:, a:b], phi[:, :, a:b]
        O = np.einsum("mi,wmj->wij", ps, ph)
        kappa = np.maximum(kappa, np.linalg.cond(O))
        Th = np.einsum("wmj,wjk->wmk", ph, np.linalg.inv(O))           # Theta = Phi O^-1
        e1 += np.einsum("na,wan->w", ps.T @ h1, Th)
        T = products(np.einsum("ma,gmi->gai", ps, L), Th)             # L~_g = Psi^T L_g
        tr = tr + np.einsum("wgaa->wg", T)
        ex += np.einsum("wgab,wgba->w", T, T)
    return e1, 0.5 * (np.sum(tr * tr, axis=1) - ex), kappa


def exact(Lt, Th):
    return np.einsum("gai,wib->wgab", Lt, Th, optimize=True)


def split3(Lt, Th, drop_lo_hi=False):
    """hi*hi + hi*lo + lo*hi of the split operands, summed exactly (Theta from FP32)."""
    Lh, Ll = split(Lt)
    th32 = Th.astype(np.complex64)
    out = 0
    for part, unit in ((th32.real, 1.0), (th32.imag, 1j)):
        Th_h, Th_l = split(part)
        t = exact(Lh, Th_h) + exact(Lh, Th_l)
        if not drop_lo_hi:
            t = t + exact(Ll, Th_h)
        out = out + unit * t
    return out


@pytest.fixture(scope="module")
def c3():
    d = build_system(**CONFIGS["C3"]["A"], coupling="moderate")
    return d, walkers(d, 6, seed=11)


def test_restatement_matches_the_oracle_local_energy(c3):
    d, phi = c3
    e1, e2, _ = energy_terms(d, phi, exact)
    o = orc.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], CONFIGS["C3"]["dt"])
    ref = orc.local_energy(o, phi)
    assert np.max(np.abs(e1 + e2 - ref) / np.abs(ref)) < 1e-10


def test_split_bf16_energy_error_sits_inside_the_gpu_bound(c3):
    d, phi = c3
    _, e2, kappa = energy_terms(d, phi, exact)
    _, e2s, _ = energy_terms(d, phi, split3)
    err = np.abs(e2s - e2)
    assert np.all(err <= 0.5 * (BOUND[0] + BOUND[1] * kappa)), (err, kappa)
    assert err.max() > 1e-9   # rounding of the split, not an exact product


def test_emulation_detects_a_dropped_split_product(c3):
    """Two products instead of three (lo*hi dropped) leave an error at the bf16 level, far
    above the three-product error: the emulation resolves the arithmetic it vouches for."""
    d, phi = c3
    _, e2, _ = energy_terms(d, phi, exact)
    _, e2s, _ = energy_terms(d, phi, split3)
    _, e2d, _ = energy_terms(d, phi, lambda Lt, Th: split3(Lt, Th, drop_lo_hi=True))
    assert np.abs(e2d - e2).max() > 20 * np.abs(e2s - e2).max()
