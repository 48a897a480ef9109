// FP32 kernels of the split-precision step (AFQMC_BF16X3): the propagator products
// (one-body half steps, Taylor exponential) and the exchange energy run in FP32 on the
// CUDA cores, roughly 60x the FP64 rate of this part, while overlaps, determinants,
// ratios, weights and Gram-Schmidt stay in FP64 and the Cholesky contractions (force
// bias, V_HS) run on the tensor cores (gemm_tc.cu).
#include "device_util.cuh"
#include "internal.h"

namespace afq {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <class T>
__device__ __forceinline__ float to_f(T v) { return (float)v; }

// C[n*ldc + m] = alpha * sum_k A[m*lda + k] * B[n*ldb + k], FP32 accumulation.
// Thread (tx, ty) owns rows m0+4tx..+3 and columns n0+4ty..+3 (float4 shared reads).
template <class TB, class TC>
__global__ void __launch_bounds__(NT) k_gemm_tn_f32(int Md, int Nd, int Kd, float alpha,
                                                    const float* __restrict__ A, int64_t lda,
                                                    const TB* __restrict__ B, int64_t ldb,
                                                    TC* __restrict__ C, int64_t ldc) {
  __shared__ __align__(16) float As[BK][BM];
  __shared__ __align__(16) float Bs[BK][BN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int r = tid >> 2, c0 = (tid & 3) * 4;
  const bool arow = (m0 + r) < Md, brow = (n0 + r) < Nd;
  const float* Ap = A + (int64_t)(m0 + r) * lda;
  const TB* Bp = B + (int64_t)(n0 + r) * ldb;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < Kd; k0 += BK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + c0 + q;
      As[c0 + q][r] = (arow && k < Kd) ? __ldg(Ap + k) : 0.f;
      Bs[c0 + q][r] = (brow && k < Kd) ? to_f(__ldg(Bp + k)) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(&As[kk][4 * tx]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][4 * ty]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int n = n0 + 4 * ty + j;
    if (n >= Nd) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = m0 + 4 * tx + i;
      if (m < Md) C[(int64_t)n * ldc + m] = (TC)(alpha * acc[i][j]);
    }
  }
}

// Taylor exponential in FP32: Phi <- sum_{m<=n} A^m Phi / m! per walker, A complex
// [M][M] (full, planar [2][Nw][M*M]).  Terms are kept in shared memory as [row][NP]
// with NP = N rounded up to 4 (zero columns); a thread owns one row i and four columns,
// so one broadcast load of A[i][j] feeds four complex MACs.
template <int OPT>
__global__ void __launch_bounds__(256) k_taylor_f32(float* __restrict__ phi, const float* __restrict__ Av,
                                                    int M, int N, int Nw, int order) {
  extern __shared__ float smf[];
  const int wk = blockIdx.x, tid = threadIdx.x;
  const int NP = (N + 3) & ~3, NG = NP / 4, NMP = M * NP;
  float* tr = smf;
  float* ti = tr + NMP;
  float* nr = ti + NMP;
  float* ni = nr + NMP;
  const int64_t plane = (int64_t)Nw * N * M, base = (int64_t)wk * N * M;
  const int64_t MM = (int64_t)M * M;
  const float* ar = Av + (int64_t)wk * MM;
  const float* ai = Av + (int64_t)Nw * MM + (int64_t)wk * MM;
  for (int e = tid; e < NMP; e += blockDim.x) {
    const int i = e / NP, b = e % NP;
    float vr = 0.f, vi = 0.f;
    if (b < N) {
      vr = phi[base + (int64_t)b * M + i];
      vi = phi[plane + base + (int64_t)b * M + i];
    }
    tr[e] = vr;
    ti[e] = vi;
  }
  __syncthreads();
  float sr[OPT][4], si[OPT][4];
#pragma unroll
  for (int q = 0; q < OPT; ++q) {
    const int o = tid + q * 256;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      sr[q][c] = (o < M * NG) ? tr[(o / NG) * NP + (o % NG) * 4 + c] : 0.f;
      si[q][c] = (o < M * NG) ? ti[(o / NG) * NP + (o % NG) * 4 + c] : 0.f;
    }
  }
  for (int m = 1; m <= order; ++m) {
    const float inv = 1.f / (float)m;
#pragma unroll
    for (int q = 0; q < OPT; ++q) {
      const int o = tid + q * 256;
      if (o < M * NG) {
        const int i = o / NG, b0 = (o % NG) * 4;
        float xr[4] = {0.f, 0.f, 0.f, 0.f}, xi[4] = {0.f, 0.f, 0.f, 0.f};
        const float* rowr = ar + (int64_t)i * M;
        const float* rowi = ai + (int64_t)i * M;
        for (int j = 0; j < M; ++j) {
          const float a_r = __ldg(rowr + j), a_i = __ldg(rowi + j);
          const float4 yr = *reinterpret_cast<const float4*>(tr + j * NP + b0);
          const float4 yi = *reinterpret_cast<const float4*>(ti + j * NP + b0);
          const float vr[4] = {yr.x, yr.y, yr.z, yr.w}, vi[4] = {yi.x, yi.y, yi.z, yi.w};
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            xr[c] = fmaf(a_r, vr[c], fmaf(-a_i, vi[c], xr[c]));
            xi[c] = fmaf(a_r, vi[c], fmaf(a_i, vr[c], xi[c]));
          }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          xr[c] *= inv;
          xi[c] *= inv;
          nr[i * NP + b0 + c] = xr[c];
          ni[i * NP + b0 + c] = xi[c];
          sr[q][c] += xr[c];
          si[q][c] += xi[c];
        }
      }
    }
    __syncthreads();
    float* t0 = tr; tr = nr; nr = t0;
    float* t1 = ti; ti = ni; ni = t1;
  }
#pragma unroll
  for (int q = 0; q < OPT; ++q) {
    const int o = tid + q * 256;
    if (o < M * NG) {
      const int i = o / NG, b0 = (o % NG) * 4;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int b = b0 + c;
        if (b < N) {
          phi[base + (int64_t)b * M + i] = sr[q][c];
          phi[plane + base + (int64_t)b * M + i] = si[q][c];
        }
      }
    }
  }
}

// Local energy with FP32 products (the exchange part dominates): same formula and
// traversal as the FP64 kernel, per-g sums in FP32, totals in FP64.
constexpr int G_CH = 4;
__global__ void __launch_bounds__(256) k_energy_f32(const double* __restrict__ theta,
                                                    const float* __restrict__ Ltil,
                                                    const double* __restrict__ htil,
                                                    double* __restrict__ eloc, int M, int N,
                                                    int n_up, int X, int Nw) {
  extern __shared__ float sme[];
  const int wk = blockIdx.x, tid = threadIdx.x, NM = N * M;
  const int nu = n_up, nd = N - n_up, nn = nu * nu + nd * nd;
  float* thr = sme;
  float* thi = thr + NM;
  float* Tr = thi + NM;
  float* Ti = Tr + G_CH * nn;
  double* red = reinterpret_cast<double*>(Ti + G_CH * nn + ((G_CH * nn) & 1));
  const int64_t plane = (int64_t)Nw * NM, base = (int64_t)wk * NM;
  double acc[4] = {0, 0, 0, 0};
  for (int e = tid; e < NM; e += blockDim.x) {
    const int n = e / M, i = e % M;
    const double vr = theta[base + e], vi = theta[plane + base + e];
    thr[i * N + n] = (float)vr;
    thi[i * N + n] = (float)vi;
    const double h = __ldg(htil + e);
    acc[0] = fma(h, vr, acc[0]);
    acc[1] = fma(h, vi, acc[1]);
  }
  __syncthreads();
  for (int g0 = 0; g0 < X; g0 += G_CH) {
    const int gc = min(G_CH, X - g0);
    for (int e = tid; e < gc * nn; e += blockDim.x) {
      const int gl = e / nn, r = e % nn;
      int a, b, n0;
      if (r < nu * nu) { a = r / nu; b = r % nu; n0 = 0; }
      else { const int r2 = r - nu * nu; a = r2 / nd; b = r2 % nd; n0 = nu; }
      const float* lrow = Ltil + ((int64_t)(g0 + gl) * N + n0 + a) * M;
      float sr = 0.f, si = 0.f;
      for (int i = 0; i < M; ++i) {
        const float l = __ldg(lrow + i);
        sr = fmaf(l, thr[i * N + n0 + b], sr);
        si = fmaf(l, thi[i * N + n0 + b], si);
      }
      Tr[e] = sr;
      Ti[e] = si;
    }
    __syncthreads();
    float ex_r = 0.f, ex_i = 0.f;
    for (int e = tid; e < gc * nn; e += blockDim.x) {
      const int gl = e / nn, r = e % nn;
      int et;
      if (r < nu * nu) { const int a = r / nu, b = r % nu; et = b * nu + a; }
      else { const int r2 = r - nu * nu; const int a = r2 / nd, b = r2 % nd; et = nu * nu + b * nd + a; }
      const float pr = Tr[e] * Tr[gl * nn + et] - Ti[e] * Ti[gl * nn + et];
      const float pi = Tr[e] * Ti[gl * nn + et] + Ti[e] * Tr[gl * nn + et];
      ex_r += pr;
      ex_i += pi;
    }
    acc[2] -= 0.5 * (double)ex_r;
    acc[3] -= 0.5 * (double)ex_i;
    for (int gl = tid; gl < gc; gl += blockDim.x) {
      float cr = 0.f, ci = 0.f;
      for (int a = 0; a < nu; ++a) { cr += Tr[gl * nn + a * nu + a]; ci += Ti[gl * nn + a * nu + a]; }
      for (int a = 0; a < nd; ++a) {
        cr += Tr[gl * nn + nu * nu + a * nd + a];
        ci += Ti[gl * nn + nu * nu + a * nd + a];
      }
      acc[0] += 0.5 * ((double)cr * cr - (double)ci * ci);
      acc[1] += (double)cr * ci;
    }
    __syncthreads();
  }
  block_sum<4>(acc, red);
  if (tid == 0) {
    eloc[wk] = acc[0] + acc[2];
    eloc[Nw + wk] = acc[1] + acc[3];
  }
}

__global__ void k_to_float(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (float)in[e];
}

int taylor_opt(int M, int N) {
  const int pairs = M * (((N + 3) & ~3) / 4);
  return (pairs + 255) / 256;
}

}  // namespace

size_t smem_taylor_f32(const Ctx& c) { return sizeof(float) * 4 * (size_t)c.M * ((c.N + 3) & ~3); }
size_t smem_energy_f32(const Ctx& c) {
  const size_t nu = c.n_up, nd = c.N - c.n_up, nn = nu * nu + nd * nd;
  return sizeof(float) * (2 * (size_t)c.N * c.M + 2 * G_CH * nn + 2) + sizeof(double) * 64;
}

cudaError_t prepare_mixed_kernels(const Ctx& c) {
  static size_t have_t = 0, have_e = 0;
  cudaError_t e;
  const size_t st = smem_taylor_f32(c), se = smem_energy_f32(c);
  if (st > have_t) {
    for (auto f : {k_taylor_f32<1>, k_taylor_f32<2>, k_taylor_f32<4>})
      if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)st)) !=
          cudaSuccess)
        return e;
    have_t = st;
  }
  if (se > have_e) {
    if ((e = cudaFuncSetAttribute(k_energy_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)se)) != cudaSuccess)
      return e;
    have_e = se;
  }
  return cudaSuccess;
}

cudaError_t gemm_f32_from_f64(int Md, int Nd, int Kd, float alpha, const float* A, int64_t lda,
                              const double* B, int64_t ldb, float* C, int64_t ldc, cudaStream_t s) {
  dim3 grid((Md + BM - 1) / BM, (Nd + BN - 1) / BN);
  if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
  k_gemm_tn_f32<double, float><<<grid, NT, 0, s>>>(Md, Nd, Kd, alpha, A, lda, B, ldb, C, ldc);
  return cudaGetLastError();
}

cudaError_t gemm_f32_to_f64(int Md, int Nd, int Kd, float alpha, const float* A, int64_t lda,
                            const float* B, int64_t ldb, double* C, int64_t ldc, cudaStream_t s) {
  dim3 grid((Md + BM - 1) / BM, (Nd + BN - 1) / BN);
  if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
  k_gemm_tn_f32<float, double><<<grid, NT, 0, s>>>(Md, Nd, Kd, alpha, A, lda, B, ldb, C, ldc);
  return cudaGetLastError();
}

cudaError_t launch_taylor_f32(const Ctx& c, float* phi32, const float* A32, cudaStream_t s) {
  const int opt = taylor_opt(c.M, c.N);
  const size_t smem = smem_taylor_f32(c);
  if (opt <= 1) k_taylor_f32<1><<<c.Nw, 256, smem, s>>>(phi32, A32, c.M, c.N, c.Nw, c.opt.taylor_order);
  else if (opt <= 2) k_taylor_f32<2><<<c.Nw, 256, smem, s>>>(phi32, A32, c.M, c.N, c.Nw, c.opt.taylor_order);
  else if (opt <= 4) k_taylor_f32<4><<<c.Nw, 256, smem, s>>>(phi32, A32, c.M, c.N, c.Nw, c.opt.taylor_order);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_energy_f32(const Ctx& c, const float* Ltil32, cudaStream_t s, int n_walkers) {
  k_energy_f32<<<n_walkers > 0 ? n_walkers : c.Nw, 256, smem_energy_f32(c), s>>>(
      c.theta, Ltil32, c.htil, c.eloc, c.M, c.N, c.n_up, c.X, c.Nw);
  return cudaGetLastError();
}

cudaError_t to_float(const double* in, float* out, int64_t n, cudaStream_t s) {
  int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 64);
  if (grid < 1) grid = 1;
  k_to_float<<<grid, 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

}  // namespace afq
