// FP64 "TN" GEMM: both operands stored with the contraction index contiguous.
//
//   C[z][n*ldc + m] = alpha * sum_k A[z][m*lda + k] * B[z][n*ldb + k]  (+ beta * C)
//
// Every Cholesky contraction of the propagation step has this form once walkers
// are stored as planar complex column blocks:
//   force bias (Eq. 9):   rhobar[(p,w)][g] = sum_(n,i) Ltil[g][(n,i)] Theta[(p,w)][(n,i)]
//   V_HS (Eq. 11):        A[(p,w)][ij]     = sum_g Lt[ij][g] U[(p,w)][g]
//   one-body half-step:   Phi'[(p,w,n)][i] = sum_j expK[i][j] Phi[(p,w,n)][j]
// (p = real/imaginary plane).  GB300's FP64 pipe (about 1 TFLOP/s measured) is
// the bound for all of them, so the kernel is a register-tiled DFMA GEMM whose
// only job is to keep that pipe busy: 64x64 CTA tile, 16-deep k slices staged
// through shared memory (transposed, so the inner loop reads contiguous rows),
// 4x4 outputs per thread, fused alpha/beta epilogue with coalesced stores.
#include "internal.h"

namespace afq {

namespace {
constexpr int BM = 64, BN = 64, BK = 16, NT = 256;
constexpr int TM = BM / 16, TN = BN / 16;

__device__ __forceinline__ void gemm_tn_body(int Md, int Nd, int Kd, double alpha,
                                             const double* __restrict__ A, int64_t lda, int64_t sA,
                                             const double* __restrict__ B, int64_t ldb, int64_t sB,
                                             double beta, double* __restrict__ C, int64_t ldc,
                                             int64_t sC) {
  __shared__ double As[2][BK][BM];
  __shared__ double Bs[2][BK][BN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t z = blockIdx.z;
  A += z * sA;
  B += z * sB;
  C += z * sC;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;

  // each thread stages 4 elements of A and 4 of B per k slice (row r, cols c0..c0+3)
  const int r = tid >> 2, c0 = (tid & 3) * 4;
  const bool arow = (m0 + r) < Md, brow = (n0 + r) < Nd;
  const double* Ap = A + (int64_t)(m0 + r) * lda;
  const double* Bp = B + (int64_t)(n0 + r) * ldb;
  double ra[4], rb[4];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + c0 + q;
      ra[q] = (arow && k < Kd) ? __ldg(Ap + k) : 0.0;
      rb[q] = (brow && k < Kd) ? __ldg(Bp + k) : 0.0;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      As[buf][c0 + q][r] = ra[q];
      Bs[buf][c0 + q][r] = rb[q];
    }
  };

  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

  fetch(0);
  stash(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < Kd; k0 += BK) {
    const bool more = (k0 + BK) < Kd;
    if (more) fetch(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (more) {
      stash(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }

#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const int n = n0 + ty + 16 * j;
    if (n >= Nd) continue;
    double* Cp = C + (int64_t)n * ldc;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int m = m0 + tx + 16 * i;
      if (m < Md) Cp[m] = (beta != 0.0) ? fma(alpha, acc[i][j], beta * Cp[m]) : alpha * acc[i][j];
    }
  }
}
// One kernel symbol per use, so profiles and launch lists name the contraction.
#define AFQ_GEMM_KERNEL(name)                                                                    \
  __global__ void __launch_bounds__(NT) name(int Md, int Nd, int Kd, double alpha,              \
                                             const double* __restrict__ A, int64_t lda, int64_t sA, \
                                             const double* __restrict__ B, int64_t ldb, int64_t sB, \
                                             double beta, double* __restrict__ C, int64_t ldc,   \
                                             int64_t sC) {                                       \
    gemm_tn_body(Md, Nd, Kd, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);                   \
  }
AFQ_GEMM_KERNEL(k_gemm_f64_generic)
AFQ_GEMM_KERNEL(k_gemm_f64_force_bias)
AFQ_GEMM_KERNEL(k_gemm_f64_vhs)
AFQ_GEMM_KERNEL(k_gemm_f64_onebody)
#undef AFQ_GEMM_KERNEL
}  // namespace

cudaError_t gemm_tn_f64(int Md, int Nd, int Kd, double alpha, const double* A, int64_t lda,
                        int64_t sA, const double* B, int64_t ldb, int64_t sB, double beta,
                        double* C, int64_t ldc, int64_t sC, int batch, cudaStream_t s,
                        GemmUse use) {
  if (Md <= 0 || Nd <= 0 || batch <= 0) return cudaSuccess;
  dim3 grid((Md + BM - 1) / BM, (Nd + BN - 1) / BN, batch);
  if (grid.y > 65535u || grid.z > 65535u) return cudaErrorInvalidConfiguration;
  auto k = use == GEMM_FORCE_BIAS ? k_gemm_f64_force_bias
           : use == GEMM_VHS      ? k_gemm_f64_vhs
           : use == GEMM_ONEBODY  ? k_gemm_f64_onebody
                                  : k_gemm_f64_generic;
  k<<<grid, NT, 0, s>>>(Md, Nd, Kd, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
  return cudaGetLastError();
}

}  // namespace afq
