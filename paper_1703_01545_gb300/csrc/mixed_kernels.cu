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
  static SmemLimits lim;
  const size_t st = smem_taylor_f32(c), se = smem_energy_f32(c);
  cudaError_t e = lim.raise(0, st, [&] {
    for (auto f : {k_taylor_f32<1>, k_taylor_f32<2>, k_taylor_f32<4>}) {
      cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)st);
      if (r != cudaSuccess) return r;
    }
    return cudaSuccess;
  });
  if (e != cudaSuccess) return e;
  return lim.raise(1, se, [&] {
    return cudaFuncSetAttribute(k_energy_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)se);
  });
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

__global__ void k_split_f32(const double* __restrict__ in, float* __restrict__ hi, float* __restrict__ lo,
                            int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float h = (float)in[e];
    hi[e] = h;
    lo[e] = (float)(in[e] - (double)h);
  }
}

cudaError_t split_f32(const double* in, float* hi, float* lo, int64_t n, cudaStream_t s) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
  k_split_f32<<<grid, 256, 0, s>>>(in, hi, lo, n);
  return cudaGetLastError();
}

cudaError_t to_float(const double* in, float* out, int64_t n, cudaStream_t s) {
  int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 64);
  if (grid < 1) grid = 1;
  k_to_float<<<grid, 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

}  // namespace afq

// ===========================================================================
// Second-generation FP32 kernels of the split-precision step.
// ===========================================================================
namespace afq {
namespace {

// Exchange + Coulomb local energy with several walkers per CTA.
//   LtT  [X][M][NPT]  float: (Psi_s^T L_g) transposed, spin blocks padded to multiples of 4
//   th   [2][Nw][N][M] float: Theta (planar)
// For each chunk of GC Cholesky vectors the CTA stages LtT for the chunk, every thread forms
// 4x4 tiles of T^s_g = Psi_s^T L_g Theta_s for one (walker, g) from float4 shared reads,
// tiles land in shared memory, and each walker's own thread group accumulates
// sum_ab T_ab T_ba and (sum_s tr T^s_g)^2.
template <int WB>
__global__ void __launch_bounds__(256) k_energy_f32_tiled(const float* __restrict__ th,
                                                          const float* __restrict__ LtT,
                                                          const double* __restrict__ htil,
                                                          double* __restrict__ eloc, int M, int N,
                                                          int n_up, int X, int Nw, int GC) {
  extern __shared__ __align__(16) float s4[];
  const int nu = n_up, nd = N - n_up;
  const int PU = (nu + 3) & ~3, PD = (nd + 3) & ~3, NPT = PU + PD;
  const int tu = PU / 4, td = PD / 4, ntiles = tu * tu + td * td;
  const int tid = threadIdx.x;
  const int w0 = blockIdx.x * WB;
  float* thr = s4;                         // [WB][M][NPT]
  float* thi = thr + WB * M * NPT;
  const int LS = M * NPT + 4;              // per-g stride: +4 floats shifts banks, keeps float4
  float* Ls = thi + WB * M * NPT;          // [GC][LS]
  const int nnp = PU * PU + PD * PD;
  const int nst = nnp + 1;                 // odd stride between (walker, g) blocks: no bank conflicts
  float* Tr = Ls + GC * LS;                // [WB][GC][nst]
  float* Ti = Tr + WB * GC * nst;
  double* red = reinterpret_cast<double*>(Ti + WB * GC * nst + ((2 * WB * GC * nst) & 1));
  const int64_t plane = (int64_t)Nw * N * M;
  // stage Theta of the CTA's walkers, spin-padded columns, zero elsewhere
  for (int e = tid; e < WB * M * NPT; e += blockDim.x) {
    const int wl = e / (M * NPT), r = e % (M * NPT), i = r / NPT, c = r % NPT;
    int n = -1;
    if (c < PU) { if (c < nu) n = c; }
    else if (c - PU < nd) n = nu + (c - PU);
    float vr = 0.f, vi = 0.f;
    const int wk = w0 + wl;
    if (n >= 0 && wk < Nw) {
      const int64_t gi = ((int64_t)wk * N + n) * M + i;
      vr = th[gi];
      vi = th[plane + gi];
    }
    thr[e] = vr;
    thi[e] = vi;
  }
  // one-body part: threads of walker group wl
  const int per_w = blockDim.x / WB;       // threads per walker in the reduction
  const int wl_me = tid / per_w, lt = tid % per_w;
  double acc[4] = {0, 0, 0, 0};            // sum for walker wl_me: E1+coul (re, im), -exch/2 (re, im)
  if (wl_me < WB && w0 + wl_me < Nw) {
    const int wk = w0 + wl_me;
    for (int e = lt; e < N * M; e += per_w) {
      const double h = __ldg(htil + e);
      const int64_t gi = (int64_t)wk * N * M + e;
      acc[0] = fma(h, (double)th[gi], acc[0]);
      acc[1] = fma(h, (double)th[plane + gi], acc[1]);
    }
  }
  __syncthreads();
  const int items = WB * GC * ntiles;
  for (int g0 = 0; g0 < X; g0 += GC) {
    const int gc = min(GC, X - g0);
    for (int e = tid; e < gc * M * NPT; e += blockDim.x)
      Ls[(e / (M * NPT)) * LS + e % (M * NPT)] = LtT[(int64_t)g0 * M * NPT + e];
    __syncthreads();
    for (int it = tid; it < items; it += blockDim.x) {
      const int wl = it / (GC * ntiles), r = it % (GC * ntiles), gl = r / ntiles, t = r % ntiles;
      if (gl >= gc) continue;
      int c0a, c0b, toff, P;
      if (t < tu * tu) { c0a = 4 * (t / tu); c0b = 4 * (t % tu); toff = 0; P = PU; }
      else { const int t2 = t - tu * tu; c0a = PU + 4 * (t2 / td); c0b = PU + 4 * (t2 % td); toff = PU * PU; P = PD; }
      float ar[4][4], ai[4][4];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) ar[x][y] = ai[x][y] = 0.f;
      const float* Lp = Ls + gl * LS + c0a;
      const float* Rp = thr + wl * M * NPT + c0b;
      const float* Ip = thi + wl * M * NPT + c0b;
      for (int i = 0; i < M; ++i) {
        const float4 l = *reinterpret_cast<const float4*>(Lp + i * NPT);
        const float4 tr = *reinterpret_cast<const float4*>(Rp + i * NPT);
        const float4 ti = *reinterpret_cast<const float4*>(Ip + i * NPT);
        const float lv[4] = {l.x, l.y, l.z, l.w}, rv[4] = {tr.x, tr.y, tr.z, tr.w},
                    iv[4] = {ti.x, ti.y, ti.z, ti.w};
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            ar[x][y] = fmaf(lv[x], rv[y], ar[x][y]);
            ai[x][y] = fmaf(lv[x], iv[y], ai[x][y]);
          }
      }
      // store tile: block-local indices (a, b) inside the spin block
      const int la = c0a - (toff ? PU : 0), lb = c0b - (toff ? PU : 0);
      float* Trp = Tr + (wl * GC + gl) * nst + toff;
      float* Tip = Ti + (wl * GC + gl) * nst + toff;
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          Trp[(la + x) * P + lb + y] = ar[x][y];
          Tip[(la + x) * P + lb + y] = ai[x][y];
        }
    }
    __syncthreads();
    if (wl_me < WB) {
      float ex_r = 0.f, ex_i = 0.f;
      for (int e = lt; e < gc * nnp; e += per_w) {
        const int gl = e / nnp, r = e % nnp;
        int et;
        if (r < PU * PU) { const int a = r / PU, b = r % PU; et = b * PU + a; }
        else { const int r2 = r - PU * PU, a = r2 / PD, b = r2 % PD; et = PU * PU + b * PD + a; }
        const float* trp = Tr + (wl_me * GC + gl) * nst;
        const float* tip = Ti + (wl_me * GC + gl) * nst;
        ex_r += trp[r] * trp[et] - tip[r] * tip[et];
        ex_i += trp[r] * tip[et] + tip[r] * trp[et];
      }
      acc[2] -= 0.5 * (double)ex_r;
      acc[3] -= 0.5 * (double)ex_i;
      for (int gl = lt; gl < gc; gl += per_w) {
        const float* trp = Tr + (wl_me * GC + gl) * nst;
        const float* tip = Ti + (wl_me * GC + gl) * nst;
        float cr = 0.f, ci = 0.f;
        for (int a = 0; a < nu; ++a) { cr += trp[a * PU + a]; ci += tip[a * PU + a]; }
        for (int a = 0; a < nd; ++a) { cr += trp[PU * PU + a * PD + a]; ci += tip[PU * PU + a * PD + a]; }
        acc[0] += 0.5 * ((double)cr * cr - (double)ci * ci);
        acc[1] += (double)cr * ci;
      }
    }
    __syncthreads();
  }
  // per-walker reduction over its per_w threads (whole warps: per_w is a multiple of 32)
#pragma unroll
  for (int q = 0; q < 4; ++q)
    for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_down_sync(0xffffffffu, acc[q], o);
  const int lane = tid & 31, wid = tid >> 5;
  if (lane == 0)
    for (int q = 0; q < 4; ++q) red[q * 8 + wid] = acc[q];
  __syncthreads();
  if (tid < WB && w0 + tid < Nw) {
    const int wpw = per_w / 32;
    double v[4] = {0, 0, 0, 0};
    for (int q = 0; q < 4; ++q)
      for (int k = 0; k < wpw; ++k) v[q] += red[q * 8 + tid * wpw + k];
    eloc[w0 + tid] = v[0] + v[2];
    eloc[Nw + w0 + tid] = v[1] + v[3];
  }
}

// LtT[g][i][c] from Ltil[g][n][i] (float64), spin-padded columns
__global__ void k_build_LtT(const double* __restrict__ Ltil, float* __restrict__ LtT, int X, int M,
                            int N, int n_up) {
  const int nu = n_up, nd = N - n_up, PU = (nu + 3) & ~3, PD = (nd + 3) & ~3, NPT = PU + PD;
  const int64_t total = (int64_t)X * M * NPT;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % NPT);
    const int64_t r = e / NPT;
    const int i = (int)(r % M);
    const int g = (int)(r / M);
    int n = -1;
    if (c < PU) { if (c < nu) n = c; }
    else if (c - PU < nd) n = nu + (c - PU);
    LtT[e] = n >= 0 ? (float)Ltil[((int64_t)g * N + n) * M + i] : 0.f;
  }
}

// Taylor exponential, A_w staged in shared memory.  A is complex symmetric, so row j of A
// is column j: the loop reads A[j][i..i+1] contiguously.  Each thread owns rows
// (2ip, 2ip+1) and columns (4bg .. 4bg+3): per j two float2 and two float4 shared loads
// feed 32 FMAs.
__global__ void __launch_bounds__(256) k_taylor_f32_smem(float* __restrict__ phi,
                                                         const float* __restrict__ Av, int M,
                                                         int N, int Nw, int order) {
  extern __shared__ __align__(16) float sm2[];
  const int wk = blockIdx.x, tid = threadIdx.x;
  const int NP = (N + 3) & ~3, NG = NP / 4, MP = (M + 1) & ~1, RH = MP / 2;
  const int64_t MM = (int64_t)M * M;
  float* Ar = sm2;                   // [M][MP]
  float* Ai = Ar + M * MP;
  float* tr = Ai + M * MP;           // [MP][NP]
  float* ti = tr + MP * NP;
  float* nr = ti + MP * NP;
  float* ni = nr + MP * NP;
  const float* ar_g = Av + (int64_t)wk * MM;
  const float* ai_g = Av + (int64_t)Nw * MM + (int64_t)wk * MM;
  for (int e = tid; e < M * MP; e += blockDim.x) {
    const int j = e / MP, i = e % MP;
    Ar[e] = i < M ? ar_g[(int64_t)j * M + i] : 0.f;
    Ai[e] = i < M ? ai_g[(int64_t)j * M + i] : 0.f;
  }
  const int64_t plane = (int64_t)Nw * N * M, base = (int64_t)wk * N * M;
  for (int e = tid; e < MP * NP; e += blockDim.x) {
    const int i = e / NP, b = e % NP;
    float vr = 0.f, vi = 0.f;
    if (b < N && i < M) {
      vr = phi[base + (int64_t)b * M + i];
      vi = phi[plane + base + (int64_t)b * M + i];
    }
    tr[e] = vr;
    ti[e] = vi;
    nr[e] = 0.f;
    ni[e] = 0.f;
  }
  __syncthreads();
  const int items = RH * NG;
  // each thread: at most 2 items (RH*NG <= 512)
  float sr[2][2][4], si[2][2][4];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int o = tid + q * 256;
    const int ip = o / NG, b0 = (o % NG) * 4;
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        sr[q][rr][c] = (o < items) ? tr[(2 * ip + rr) * NP + b0 + c] : 0.f;
        si[q][rr][c] = (o < items) ? ti[(2 * ip + rr) * NP + b0 + c] : 0.f;
      }
  }
  for (int m = 1; m <= order; ++m) {
    const float inv = 1.f / (float)m;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int o = tid + q * 256;
      if (o < items) {
        const int ip = o / NG, b0 = (o % NG) * 4;
        float xr[2][4], xi[2][4];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr)
#pragma unroll
          for (int c = 0; c < 4; ++c) xr[rr][c] = xi[rr][c] = 0.f;
        for (int j = 0; j < M; ++j) {
          const float2 a_r = *reinterpret_cast<const float2*>(Ar + j * MP + 2 * ip);
          const float2 a_i = *reinterpret_cast<const float2*>(Ai + j * MP + 2 * ip);
          const float4 yr = *reinterpret_cast<const float4*>(tr + j * NP + b0);
          const float4 yi = *reinterpret_cast<const float4*>(ti + j * NP + b0);
          const float Rr[2] = {a_r.x, a_r.y}, Ri[2] = {a_i.x, a_i.y};
          const float vr[4] = {yr.x, yr.y, yr.z, yr.w}, vi[4] = {yi.x, yi.y, yi.z, yi.w};
#pragma unroll
          for (int rr = 0; rr < 2; ++rr)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              xr[rr][c] = fmaf(Rr[rr], vr[c], fmaf(-Ri[rr], vi[c], xr[rr][c]));
              xi[rr][c] = fmaf(Rr[rr], vi[c], fmaf(Ri[rr], vr[c], xi[rr][c]));
            }
        }
#pragma unroll
        for (int rr = 0; rr < 2; ++rr)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float a = xr[rr][c] * inv, b = xi[rr][c] * inv;
            nr[(2 * ip + rr) * NP + b0 + c] = a;
            ni[(2 * ip + rr) * NP + b0 + c] = b;
            sr[q][rr][c] += a;
            si[q][rr][c] += b;
          }
      }
    }
    __syncthreads();
    float* t0 = tr; tr = nr; nr = t0;
    float* t1 = ti; ti = ni; ni = t1;
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int o = tid + q * 256;
    if (o < items) {
      const int ip = o / NG, b0 = (o % NG) * 4;
#pragma unroll
      for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int i = 2 * ip + rr, b = b0 + c;
          if (i < M && b < N) {
            phi[base + (int64_t)b * M + i] = sr[q][rr][c];
            phi[plane + base + (int64_t)b * M + i] = si[q][rr][c];
          }
        }
    }
  }
}

}  // namespace

size_t smem_energy_tiled(const Ctx& c, int GC, int WB) {
  const int nu = c.n_up, nd = c.N - c.n_up, PU = (nu + 3) & ~3, PD = (nd + 3) & ~3, NPT = PU + PD;
  const size_t nst = (size_t)PU * PU + (size_t)PD * PD + 1;
  return sizeof(float) * (2 * (size_t)WB * c.M * NPT + (size_t)GC * ((size_t)c.M * NPT + 4) +
                          2 * WB * GC * nst + 2) +
         sizeof(double) * 40;
}

int energy_gc(const Ctx& c, int WB) {
  const int nu = c.n_up, nd = c.N - c.n_up, PU = (nu + 3) & ~3, PD = (nd + 3) & ~3;
  const int ntiles = (PU / 4) * (PU / 4) + (PD / 4) * (PD / 4);
  int gc = 256 / (WB * ntiles);
  if (gc < 1) gc = 1;
  while (gc > 1 && smem_energy_tiled(c, gc, WB) > 200 * 1024) --gc;
  return gc;
}

bool energy_wb_ok(const Ctx& c, int WB) { return smem_energy_tiled(c, energy_gc(c, WB), WB) <= 200 * 1024; }

size_t smem_taylor_smem(const Ctx& c) {
  const size_t NP = (c.N + 3) & ~3, MP = (c.M + 1) & ~1;
  return sizeof(float) * (2 * (size_t)c.M * MP + 4 * MP * NP);
}

bool taylor_smem_ok(const Ctx& c) {
  const int NP = (c.N + 3) & ~3, MP = (c.M + 1) & ~1;
  return smem_taylor_smem(c) <= 200 * 1024 && (MP / 2) * (NP / 4) <= 512;
}

cudaError_t prepare_mixed_kernels2(const Ctx& c) {
  static SmemLimits lim;
  cudaError_t e;
  const int wbs[3] = {2, 4, 8};
  for (int q = 0; q < 3; ++q) {
    if (!energy_wb_ok(c, wbs[q])) continue;
    const size_t se = smem_energy_tiled(c, energy_gc(c, wbs[q]), wbs[q]);
    auto f = q == 0 ? k_energy_f32_tiled<2> : q == 1 ? k_energy_f32_tiled<4> : k_energy_f32_tiled<8>;
    e = lim.raise(q, se, [&] {
      return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)se);
    });
    if (e != cudaSuccess) return e;
  }
  if (taylor_smem_ok(c)) {
    const size_t st = smem_taylor_smem(c);
    e = lim.raise(3, st, [&] {
      return cudaFuncSetAttribute(k_taylor_f32_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)st);
    });
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t build_LtT(const Ctx& c, float* LtT, cudaStream_t s) {
  const int nu = c.n_up, nd = c.N - c.n_up, NPT = ((nu + 3) & ~3) + ((nd + 3) & ~3);
  const int64_t total = (int64_t)c.X * c.M * NPT;
  int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 64);
  k_build_LtT<<<grid < 1 ? 1 : grid, 256, 0, s>>>(c.Ltil, LtT, c.X, c.M, c.N, c.n_up);
  return cudaGetLastError();
}

int64_t LtT_size(const Ctx& c) {
  const int nu = c.n_up, nd = c.N - c.n_up, NPT = ((nu + 3) & ~3) + ((nd + 3) & ~3);
  return (int64_t)c.X * c.M * NPT;
}

cudaError_t launch_energy_tiled(const Ctx& c, const float* theta32, const float* LtT,
                                cudaStream_t s, int n_walkers, int wb) {
  const int nw = n_walkers > 0 ? n_walkers : c.Nw;
  int WB = wb > 0 ? wb : (c.tune_energy_wb > 0 ? c.tune_energy_wb : 4);
  if (!energy_wb_ok(c, WB)) WB = 2;
  const int GC = energy_gc(c, WB);
  const size_t sm = smem_energy_tiled(c, GC, WB);
  const int grid = (nw + WB - 1) / WB;
  if (WB == 2)
    k_energy_f32_tiled<2><<<grid, 256, sm, s>>>(theta32, LtT, c.htil, c.eloc, c.M, c.N, c.n_up, c.X, nw, GC);
  else if (WB == 8)
    k_energy_f32_tiled<8><<<grid, 256, sm, s>>>(theta32, LtT, c.htil, c.eloc, c.M, c.N, c.n_up, c.X, nw, GC);
  else
    k_energy_f32_tiled<4><<<grid, 256, sm, s>>>(theta32, LtT, c.htil, c.eloc, c.M, c.N, c.n_up, c.X, nw, GC);
  return cudaGetLastError();
}

bool energy_variant_ok(const Ctx& c, int wb) { return energy_wb_ok(c, wb); }
bool taylor_variant_ok(const Ctx& c, int v) {
  return v == 4 ? (propagate_tcl_ok(c) && c.tcl_maps != nullptr)
       : v == 3 ? propagate_tc_ok(c) : v == 2 ? propagate_f32_ok(c) : v == 1 ? taylor_smem_ok(c) : v == 0;
}

int propagation_variant(const Ctx& c) {
  if (c.tune_taylor_smem >= 0 && taylor_variant_ok(c, c.tune_taylor_smem)) return c.tune_taylor_smem;
  for (int v : {3, 4, 2, 1}) if (taylor_variant_ok(c, v)) return v;
  return 0;
}

cudaError_t vhs_launch(const Ctx& c, int pv, cudaStream_t s) {
  const int64_t MM = (int64_t)c.M * c.M;
  if (pv == 4) {
    SplitOut so;
    so.hi = c.tcl_ahi;
    so.lo = c.tcl_alo;
    so.M = c.M;
    so.Mp = propagate_tcl_mp(c.M);
    so.ld = (int64_t)c.M * so.Mp;
    if (c.tc_Ltri) {   // the lower-triangle blocks only, the mirror half written transposed
      so.tri = 1;
      return gemm_bf16x3_split_out(*c.tc_Ltri, *c.tc_U, vhs_tri_rows(c.M), 2 * c.Nw, 1.0f, so,
                                   c.d_tc_err, s);
    }
    return gemm_bf16x3_split_out(*c.tc_L, *c.tc_U, (int)MM, 2 * c.Nw, 1.0f, so, c.d_tc_err, s);
  }
  return gemm_bf16x3(*c.tc_L, *c.tc_U, (int)MM, 2 * c.Nw, 1.0f, c.Avhs32, MM, c.d_tc_err, s);
}

cudaError_t launch_propagation(const Ctx& c, int variant, double* out, float* out32, cudaStream_t s) {
  if (variant == 4) return launch_propagate_tcl(c, out, out32, s);
  if (variant == 3) return launch_propagate_tc(c, out, out32, s);
  if (variant == 2) return launch_propagate_f32(c, out, out32, s);
  const int M = c.M, cols = 2 * c.Nw * c.N;
  cudaError_t e = gemm_f32_from_f64(M, cols, M, 1.0f, c.expK32, M, c.phi, M, c.phi32, M, s);
  if (e == cudaSuccess) e = launch_taylor_f32_variant(c, c.phi32, c.Avhs32, s, variant);
  if (e == cudaSuccess) e = gemm_f32_to_f64(M, cols, M, 1.0f, c.expK32, M, c.phi32, M, out, M, s);
  return e;
}

cudaError_t launch_taylor_f32_variant(const Ctx& c, float* phi32, const float* A32, cudaStream_t s,
                                      int use_smem) {
  if (!use_smem || !taylor_smem_ok(c)) return launch_taylor_f32(c, phi32, A32, s);
  k_taylor_f32_smem<<<c.Nw, 256, smem_taylor_smem(c), s>>>(phi32, A32, c.M, c.N, c.Nw,
                                                           c.opt.taylor_order);
  return cudaGetLastError();
}

cudaError_t launch_taylor_f32_best(const Ctx& c, float* phi32, const float* A32, cudaStream_t s) {
  if (c.tune_taylor_smem == 0 || !taylor_smem_ok(c)) return launch_taylor_f32(c, phi32, A32, s);
  k_taylor_f32_smem<<<c.Nw, 256, smem_taylor_smem(c), s>>>(phi32, A32, c.M, c.N, c.Nw,
                                                           c.opt.taylor_order);
  return cudaGetLastError();
}

}  // namespace afq
