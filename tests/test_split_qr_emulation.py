"""CPU emulation of the split path's orthonormalisation (Cholesky QR in FP32, Sec. II.D) on
walkers the oracle propagated at the C3 shape, against the bounds the GPU test of that kernel
uses (`test_cholesky_qr_orthonormalises_and_lowers_log_overlap`).

The kernel reads the walker rounded to FP32, sums the Gram matrix S = Phi_s^H Phi_s of each
spin block in FP32 (four partial sums over every fourth orbital, combined pairwise), factorises
S = R^H R in FP32, forms Q = Phi_s R^-1 by forward substitution in FP32 and lowers log O by the
FP64 sum of log R_jj over that FP32 diagonal.  The emulation takes the same steps in the same
order in numpy float32, rounding every product and every sum (the kernel's fused multiply-adds
round once where this rounds twice, so its errors are at most of this size).  The errors must
sit well inside the GPU test's bounds: Q^H Q - I and Q - Q_MGS below 5e-6, log O against an FP64
recomputation below 1e-5.
"""
import numpy as np
import pytest

from oracle import afqmc as orc
from synthetic import CONFIGS, build_system, explicit_fields

F = np.float32
BOUND_Q = 5e-6       # the GPU test's bound on Q^H Q - I and on Q - Q_MGS
BOUND_LOGO = 1e-5    # the GPU test's bound on log O against a recomputation


def gram_fp32(xr, xi):
    """S[a][b] = sum_i conj(x_ia) x_ib over four interleaved partial sums, in FP32."""
    nw, M, n = xr.shape
    parts = []
    for part in range(4):
        sr = np.zeros((nw, n, n), F)
        si = np.zeros((nw, n, n), F)
        for i in range(part, M, 4):
            ar, ai = xr[:, i, :, None], xi[:, i, :, None]
            br, bi = xr[:, i, None, :], xi[:, i, None, :]
            sr = F(sr + F(ai * bi))
            sr = F(sr + F(ar * br))
            si = F(si - F(ai * br))
            si = F(si + F(ar * bi))
        parts.append((sr, si))
    (r0, i0), (r1, i1), (r2, i2), (r3, i3) = parts
    return F(F(r0 + r1) + F(r2 + r3)), F(F(i0 + i1) + F(i2 + i3))


def cholesky_fp32(sr, si):
    """S = R^H R, R upper triangular with a positive diagonal, column step by column step."""
    Rr, Ri = sr.copy(), si.copy()
    n = Rr.shape[1]
    for k in range(n):
        d = np.sqrt(Rr[:, k, k]).astype(F)
        inv = F(F(1) / d)
        Rr[:, k, k + 1:] = F(Rr[:, k, k + 1:] * inv[:, None])
        Ri[:, k, k + 1:] = F(Ri[:, k, k + 1:] * inv[:, None])
        Rr[:, k, k], Ri[:, k, k] = d, F(0)
        for l in range(k + 1, n):
            rr, ri = Rr[:, k, l], Ri[:, k, l]
            for m in range(k + 1, l + 1):   # S_ml -= conj(R_km) R_kl
                ar, ai = Rr[:, k, m], Ri[:, k, m]
                Rr[:, m, l] = F(Rr[:, m, l] - F(F(ar * rr) + F(ai * ri)))
                Ri[:, m, l] = F(Ri[:, m, l] - F(F(ar * ri) - F(ai * rr)))
    return np.triu(Rr), np.triu(Ri)


def q_fp32(xr, xi, Rr, Ri):
    """Q = Phi R^-1 along every orbital row: q_j = (x_j - sum_{k<j} q_k R_kj) / R_jj."""
    qr, qi = xr.copy(), xi.copy()
    n = xr.shape[2]
    for j in range(n):
        tr, ti = qr[:, :, j].copy(), qi[:, :, j].copy()
        for k in range(j):
            rv_r, rv_i = Rr[:, None, k, j], Ri[:, None, k, j]
            tr = F(tr - F(F(qr[:, :, k] * rv_r) - F(qi[:, :, k] * rv_i)))
            ti = F(ti - F(F(qr[:, :, k] * rv_i) + F(qi[:, :, k] * rv_r)))
        inv = F(F(1) / Rr[:, j, j])[:, None]
        qr[:, :, j], qi[:, :, j] = F(tr * inv), F(ti * inv)
    return qr, qi


@pytest.fixture(scope="module")
def propagated():
    d = build_system(**CONFIGS["C3"]["B"], coupling="moderate")
    o = orc.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], CONFIGS["C3"]["dt"])
    nw = 4
    wk = orc.Walkers(o, nw)
    x = explicit_fields(5, nw, d["X"], seed=23)
    for t in range(5):
        orc.propagate(o, wk, x[t])
    assert wk.alive.all()
    return o, wk


def test_fp32_cholesky_qr_errors_sit_inside_the_gpu_bounds(propagated):
    o, wk = propagated
    phi = wk.phi
    Q = np.empty_like(phi)
    logdet = np.zeros(phi.shape[0])
    for a, b in o.spins:
        x = phi[:, :, a:b].astype(np.complex64)
        xr, xi = np.ascontiguousarray(x.real), np.ascontiguousarray(x.imag)
        sr, si = gram_fp32(xr, xi)
        Rr, Ri = cholesky_fp32(sr, si)
        assert np.all(np.abs(Ri[:, np.arange(b - a), np.arange(b - a)]) == 0)
        qr, qi = q_fp32(xr, xi, Rr, Ri)
        Q[:, :, a:b] = qr.astype(np.float64) + 1j * qi.astype(np.float64)
        logdet += np.log(np.diagonal(Rr, axis1=1, axis2=2).astype(np.float64)).sum(axis=1)
    err_gram = err_mgs = 0.0
    for a, b in o.spins:
        q = Q[:, :, a:b]
        gram = np.einsum("wia,wib->wab", q.conj(), q)
        err_gram = max(err_gram, np.abs(gram - np.eye(b - a)).max())
        err_mgs = max(err_mgs, np.abs(q - orc.modified_gram_schmidt(phi[:, :, a:b])).max())
    err_logo = np.abs(np.exp(wk.logO - logdet - orc.overlap(o, Q)) - 1).max()
    # the emulated errors: a few 1e-7 against bounds of 5e-6 and 1e-5
    assert err_gram < BOUND_Q / 4, err_gram
    assert err_mgs < BOUND_Q / 4, err_mgs
    assert err_logo < BOUND_LOGO / 4, err_logo
    # and they are FP32 rounding, not an exact factorisation: above the FP64 level
    assert err_gram > 1e-9


def test_emulation_detects_a_dropped_conjugate(propagated):
    """The emulation is sensitive to the arithmetic it checks: a Gram matrix without the
    conjugate (S = Phi^T Phi) no longer gives an orthonormal Q."""
    o, wk = propagated
    a, b = o.spins[0]
    x = wk.phi[:, :, a:b].astype(np.complex64)
    xr, xi = np.ascontiguousarray(x.real), np.ascontiguousarray(x.imag)
    sr, si = gram_fp32(xr, xi)
    sr_bad = F(sr - F(2) * gram_fp32(np.zeros_like(xr), xi)[0])   # drops +xi*xi: Re(x^T x)
    with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
        Rr, Ri = cholesky_fp32(sr_bad, si)
        qr, qi = q_fp32(xr, xi, Rr, Ri)
    q = qr.astype(np.float64) + 1j * qi.astype(np.float64)
    gram = np.einsum("wia,wib->wab", q.conj(), q)
    err = np.abs(gram - np.eye(b - a)).max()
    # either the wrong matrix is not positive definite (NaN) or Q is far from orthonormal
    assert not np.isfinite(err) or err > 100 * BOUND_Q, err
