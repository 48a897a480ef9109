"""The library's contraction kernels on their own, against numpy float64 products.

impl 0 (FP64 kernel) must agree to rounding; impl 1 (split-BF16 tcgen05 kernel: hi/lo
operands, hi*hi + hi*lo + lo*hi in FP32) must stay within a bound derived from its
arithmetic: each operand is represented to 2^-17 relative (bf16 hi + bf16 lo), the
dropped lo*lo term is below 2^-18 of a product, and FP32 accumulation adds K 2^-24;
elementwise |C - C_ref| <= (2^-15 + K 2^-23) (|A| |B|^T).
"""
import ctypes

import numpy as np
import pytest

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

# the last two have >= 2 x 152 output tiles of 128 x 256, so they run the persistent kernel
# (the V_HS shape of the 64-orbital workload, and a ragged one)
SHAPES = [(320, 4096, 1024), (4096, 512, 320), (70, 140, 100), (24, 256, 24), (128, 128, 64),
          (1000, 300, 950), (4096, 4096, 320), (4000, 2560, 200)]


def run(lib, impl, A, B, alpha=1.0):
    Md, K = A.shape
    Nd = B.shape[0]
    C = np.empty((Nd, Md))
    code = lib.afqmc_test_gemm(impl, Md, Nd, K, A.ctypes.data, B.ctypes.data, alpha,
                               C.ctypes.data, None)
    return code, C


@pytest.mark.parametrize("Md,Nd,K", SHAPES)
def test_contraction_kernels_against_numpy(Md, Nd, K):
    need_gpu()
    from paper_1703_01545_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(Md + Nd + K)
    A = rng.standard_normal((Md, K)) * np.exp(rng.uniform(-3, 1, (Md, 1)))
    B = rng.standard_normal((Nd, K)) * 0.07
    ref = 0.7 * (B @ A.T)
    bound = (2.0 ** -15 + K * 2.0 ** -23) * 0.7 * (np.abs(B) @ np.abs(A).T)
    code, C0 = run(lib, 0, A, B, 0.7)
    assert code == 0
    np.testing.assert_allclose(C0, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    code, C1 = run(lib, 1, A, B, 0.7)
    assert code == 0, code
    err = np.abs(C1 - ref)
    assert np.all(err <= bound), (err / bound).max()
    # far better than one BF16 product: the split really carries the low bits
    assert np.median(err / np.maximum(np.abs(ref), 1e-300)) < 1e-4


def test_bounded_wait_expires_cleanly_and_context_survives():
    """Failure detection without a GPU fault: a wait on a barrier that nothing completes
    expires (20 ms), the kernel reports it, frees its tensor memory and returns; the same
    process then runs a normal tensor-core GEMM correctly."""
    need_gpu()
    from paper_1703_01545_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(5)
    A = rng.standard_normal((128, 64))
    B = rng.standard_normal((128, 64))
    code, _ = run(lib, 2, A, B)
    assert code == 5          # AFQMC_ERR_TIMEOUT
    code, C = run(lib, 1, A, B)
    assert code == 0
    ref = B @ A.T
    assert np.all(np.abs(C - ref) <= (2.0 ** -15 + 64 * 2.0 ** -23) * (np.abs(B) @ np.abs(A).T))
