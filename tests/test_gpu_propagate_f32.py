"""Fused FP32 propagator of the split-precision step (e^{-dt K/2} e^A e^{-dt K/2} per walker in
one kernel) against the three-launch form (FP32 GEMM, Taylor kernel, FP32 GEMM).

Both are FP32 evaluations of the same products in different summation orders, so after a
few steps on the same fields the walkers agree to FP32 rounding (amplified by the
propagation), far below the split-precision path's error against FP64.  Shapes cover one to
three work tiles per thread (M = 8 .. 96), orbital counts that are not multiples of four, and
a walker count that is not a multiple of anything in particular.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, system_data
from synthetic import make_hamiltonian, scf_trial, CONFIGS, explicit_fields

pytestmark = pytest.mark.gpu


def run(afq, d, nw, dt, fields, variant):
    s = afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=dt, n_walkers=nw,
                   precision=afq.BF16X3, autotune=False)
    s.select_kernel(afq.K_TAYLOR, variant)
    s.propagate(len(fields), fields)
    st = s.state()
    info = s.info()
    s.close()
    return st, info


@pytest.mark.parametrize("cfg,which,coupling,nw", [
    ("C1", "A", 1.0, 33),
    ("C1", "B", 1.0, 17),            # 2/1: N = 3, padded to 4 columns
    ("C2", "B", "moderate", 101),    # M = 64, N = 15: one tile per thread
    ("C5", "A", "moderate", 40),     # M = 96, N = 24: three tiles per thread
])
def test_fused_propagator_matches_three_launch_form(cfg, which, coupling, nw):
    afq = need_gpu()
    d = system_data(cfg, which, coupling)
    dt = CONFIGS[cfg]["dt"]
    fields = explicit_fields(5, nw, d["X"], seed=5)
    fused, info = run(afq, d, nw, dt, fields, 2)
    assert info.tuned_taylor_smem == 2
    ref, _ = run(afq, d, nw, dt, fields, 1)
    live = fused["alive"] & ref["alive"]
    assert live.sum() >= nw - 1
    scale = np.abs(ref["phi"][live]).max()
    assert np.abs(fused["phi"][live] - ref["phi"][live]).max() < 1e-4 * scale
    np.testing.assert_allclose(fused["w"].real[live], ref["w"].real[live], rtol=1e-4)


@pytest.mark.parametrize("cfg,which,coupling,nw", [
    ("C1", "A", 1.0, 33),            # M = 8 padded to 64, N = 4 padded to 8
    ("C1", "B", 1.0, 470),           # N = 3; more walkers than resident CTAs (persistent loop)
    ("C2", "A", "moderate", 301),    # M = 64, N = 16
    ("C2", "B", "moderate", 64),     # N = 15
])
def test_tensor_core_propagator_matches_fp32(cfg, which, coupling, nw):
    """Variant 3 (split-BF16 tcgen05 rounds) against the FP32 fused kernel: the Taylor products
    carry ~2^-16 relative error of |A| |T| per step, so after 5 steps the walkers agree to
    ~1e-4 of their size."""
    afq = need_gpu()
    d = system_data(cfg, which, coupling)
    dt = CONFIGS[cfg]["dt"]
    fields = explicit_fields(5, nw, d["X"], seed=6)
    tc, info = run(afq, d, nw, dt, fields, 3)
    assert info.tuned_taylor_smem == 3
    ref, _ = run(afq, d, nw, dt, fields, 2)
    live = tc["alive"] & ref["alive"]
    assert live.sum() >= nw - 2
    scale = np.abs(ref["phi"][live]).max()
    err = np.abs(tc["phi"][live] - ref["phi"][live]).max() / scale
    assert err < 5e-4, err
    np.testing.assert_allclose(tc["w"].real[live], ref["w"].real[live], rtol=2e-3)


def test_tensor_core_propagator_refuses_large_shapes():
    """Variant 3 takes M <= 64 and N <= 16, variant 4 M <= 256 and N <= 32."""
    afq = need_gpu()
    d = system_data("C5", "A", "moderate")
    s = afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=0.005, n_walkers=8,
                   precision=afq.BF16X3, autotune=False)
    with pytest.raises(RuntimeError):
        s.select_kernel(afq.K_TAYLOR, 3)
    s.select_kernel(afq.K_TAYLOR, 4)            # M = 96, 12 + 12 columns
    assert s.info().tuned_taylor_smem == 4
    s.close()
    h1, L = make_hamiltonian(40, 8, 5)
    tr, _, _ = scf_trial(h1, L, 17, 17)
    big = afq.System(h1, L, tr, 17, 17, dt=0.005, n_walkers=4, precision=afq.BF16X3,
                     autotune=False)
    with pytest.raises(RuntimeError):
        big.select_kernel(afq.K_TAYLOR, 4)       # 34 occupied columns
    big.close()


@pytest.mark.parametrize("variant", [3, 4])
def test_dead_walkers_keep_their_state_with_in_place_propagation(variant):
    """The tensor-core propagators write live walkers in place and skip dead ones (killed by the
    cos cut, Sec. II.B): a dead walker's Phi and weight stay bit for bit as they were, and the
    mixed energy stays finite."""
    afq = need_gpu()
    d = system_data("C1", "A")
    nw = 64
    s = afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=0.1, n_walkers=nw,
                   precision=afq.BF16X3, fb_cap=0.3, autotune=False)
    s.select_kernel(afq.K_TAYLOR, variant)
    fields = explicit_fields(30, nw, d["X"], seed=41)
    s.propagate(20, fields[:20])
    s.orthonormalise()
    st1 = s.state()
    dead = ~st1["alive"]
    assert dead.any() and not dead.all()
    s.propagate(10, fields[20:])
    s.orthonormalise()
    st2 = s.state()
    _, em, _ = s.energy()
    s.close()
    assert np.array_equal(st2["phi"][dead], st1["phi"][dead])
    assert np.array_equal(st2["w"][dead], st1["w"][dead])
    assert not st2["alive"][dead].any()
    assert np.all(np.isfinite(em))
    live = st2["alive"]
    assert np.abs(st2["phi"][live] - st1["phi"][live]).max() > 0
