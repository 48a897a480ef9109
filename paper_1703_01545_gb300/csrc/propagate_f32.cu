// Fused one-step propagator of the split-precision path (Eq. 11 with the Taylor exponential):
//   Phi' = e^{-dt K/2} [ sum_{n=0}^{order} A^n / n! ] e^{-dt K/2} Phi
// for one walker per CTA, entirely in shared memory: the walker (FP64 in global, FP32 here),
// its complex symmetric A (from the V_HS contraction) and two term buffers.  Every product
// is a register-tiled SIMT loop: a thread owns 2 rows x 4 columns (8 complex outputs) and
// per index j reads A (or e^{-dt K/2}) for its two rows as a float2 and the term's row j for
// its four columns as a float4, i.e. 4 shared loads per 32 FMAs, the loads of a warp being
// broadcasts of one 64-byte segment each.  A and e^{-dt K/2} are symmetric, so their row j
// is read where the product needs column j.  The result is written as FP64 (the walker) and
// as FP32 (for the overlap kernel), coalesced through shared memory.
// Replaces, in one launch, the two one-body FP32 GEMMs and the Taylor kernel.
#include <algorithm>
#include <cstdint>

#include "internal.h"

namespace afq {
namespace {

constexpr int kPT = 128;   // threads per walker

// acc[r][c] (re, im) += sum_j A[j][2ip + r] T[j][b0 + c] for a complex A (ai != null) or a
// real one (ai == null); A rows have stride lda (floats), T rows stride NP.
template <bool CPLX>
__device__ __forceinline__ void tile_product(const float* __restrict__ ar, const float* __restrict__ ai,
                                             int lda, const float* __restrict__ tr,
                                             const float* __restrict__ ti, int NP, int K,
                                             float (&xr)[2][4], float (&xi)[2][4]) {
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) xr[r][c] = xi[r][c] = 0.f;
#pragma unroll 4
  for (int j = 0; j < K; ++j) {
    const float2 a_r = *reinterpret_cast<const float2*>(ar);
    const float4 yr = *reinterpret_cast<const float4*>(tr);
    const float4 yi = *reinterpret_cast<const float4*>(ti);
    const float R[2] = {a_r.x, a_r.y};
    const float Vr[4] = {yr.x, yr.y, yr.z, yr.w}, Vi[4] = {yi.x, yi.y, yi.z, yi.w};
    if (CPLX) {
      const float2 a_i = *reinterpret_cast<const float2*>(ai);
      const float I[2] = {a_i.x, a_i.y};
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          xr[r][c] = fmaf(R[r], Vr[c], fmaf(-I[r], Vi[c], xr[r][c]));
          xi[r][c] = fmaf(R[r], Vi[c], fmaf(I[r], Vr[c], xi[r][c]));
        }
      ai += lda;
    } else {
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          xr[r][c] = fmaf(R[r], Vr[c], xr[r][c]);
          xi[r][c] = fmaf(R[r], Vi[c], xi[r][c]);
        }
    }
    ar += lda;
    tr += NP;
    ti += NP;
  }
}

// IPT: work items (2-row x 4-column tiles) per thread, ceil((M/2) (NP/4) / 128).
template <int IPT>
__global__ void __launch_bounds__(kPT) k_propagate_f32(const double* __restrict__ phi_in,
                                                       const float* __restrict__ Av,
                                                       const float* __restrict__ expK,
                                                       double* __restrict__ phi_out,
                                                       float* __restrict__ phi_out32, int M, int N,
                                                       int Nw, int order) {
  extern __shared__ __align__(16) float sp[];
  const int wk = blockIdx.x, tid = threadIdx.x;
  const int NP = (N + 3) & ~3, NG = NP / 4, RH = M / 2, items = RH * NG;
  const int64_t MM = (int64_t)M * M, NM = (int64_t)N * M;
  float* Ar = sp;                       // A[j][i], row stride M (A symmetric)
  float* Ai = Ar + MM;
  float* t0r = Ai + MM;                 // term buffers [M][NP]
  float* t0i = t0r + M * NP;
  float* t1r = t0i + M * NP;
  float* t1i = t1r + M * NP;
  const float* ag_r = Av + (int64_t)wk * MM;
  const float* ag_i = Av + (int64_t)Nw * MM + (int64_t)wk * MM;
  for (int64_t e = tid; e < MM; e += kPT) {
    Ar[e] = ag_r[e];
    Ai[e] = ag_i[e];
  }
  const int64_t plane = (int64_t)Nw * NM, base = (int64_t)wk * NM;
  for (int e = tid; e < M * NP; e += kPT) {    // zero the padding columns of t1
    const int b = e % NP;
    if (b >= N) t1r[e] = t1i[e] = 0.f;
  }
  for (int64_t e = tid; e < NM; e += kPT) {    // coalesced read, [i][b] in shared memory
    const int b = (int)(e / M), i = (int)(e % M);
    t1r[i * NP + b] = (float)phi_in[base + e];
    t1i[i * NP + b] = (float)phi_in[plane + base + e];
  }
  __syncthreads();

  float sr[IPT][2][4], si[IPT][2][4];
  float xr[2][4], xi[2][4];
  // Phi1 = e^{-dt K/2} Phi  -> t0, running sum S = Phi1
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const int o = tid + q * kPT;
    if (o < items) {
      const int ip = o / NG, b0 = (o % NG) * 4;
      tile_product<false>(expK + 2 * ip, nullptr, M, t1r + b0, t1i + b0, NP, M, xr, xi);
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          t0r[(2 * ip + r) * NP + b0 + c] = sr[q][r][c] = xr[r][c];
          t0i[(2 * ip + r) * NP + b0 + c] = si[q][r][c] = xi[r][c];
        }
    }
  }
  __syncthreads();
  // Taylor terms T_n = A T_{n-1} / n, S += T_n
  float *cr = t0r, *ci = t0i, *nr = t1r, *ni = t1i;
  for (int n = 1; n <= order; ++n) {
    const float inv = 1.f / (float)n;
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
      const int o = tid + q * kPT;
      if (o < items) {
        const int ip = o / NG, b0 = (o % NG) * 4;
        tile_product<true>(Ar + 2 * ip, Ai + 2 * ip, M, cr + b0, ci + b0, NP, M, xr, xi);
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float vr = xr[r][c] * inv, vi = xi[r][c] * inv;
            nr[(2 * ip + r) * NP + b0 + c] = vr;
            ni[(2 * ip + r) * NP + b0 + c] = vi;
            sr[q][r][c] += vr;
            si[q][r][c] += vi;
          }
      }
    }
    __syncthreads();
    float* t = cr; cr = nr; nr = t;
    t = ci; ci = ni; ni = t;
  }
  // Phi2 = S -> shared (cr is free: its term has been consumed), then Phi' = e^{-dt K/2} Phi2
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const int o = tid + q * kPT;
    if (o < items) {
      const int ip = o / NG, b0 = (o % NG) * 4;
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          cr[(2 * ip + r) * NP + b0 + c] = sr[q][r][c];
          ci[(2 * ip + r) * NP + b0 + c] = si[q][r][c];
        }
    }
  }
  __syncthreads();
  // result tiles go to nr as [b][i] (row stride M), so the global write below is coalesced
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const int o = tid + q * kPT;
    if (o < items) {
      const int ip = o / NG, b0 = (o % NG) * 4;
      tile_product<false>(expK + 2 * ip, nullptr, M, cr + b0, ci + b0, NP, M, xr, xi);
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (b0 + c < N) {
          *reinterpret_cast<float2*>(nr + (b0 + c) * M + 2 * ip) = make_float2(xr[0][c], xr[1][c]);
          *reinterpret_cast<float2*>(ni + (b0 + c) * M + 2 * ip) = make_float2(xi[0][c], xi[1][c]);
        }
    }
  }
  __syncthreads();
  for (int64_t e = tid; e < NM; e += kPT) {
    const float vr = nr[e], vi = ni[e];
    phi_out[base + e] = (double)vr;
    phi_out[plane + base + e] = (double)vi;
    if (phi_out32) {
      phi_out32[base + e] = vr;
      phi_out32[plane + base + e] = vi;
    }
  }
}

}  // namespace

size_t smem_propagate_f32(const Ctx& c) {
  const size_t NP = (c.N + 3) & ~3;
  return sizeof(float) * (2 * (size_t)c.M * c.M + 4 * (size_t)c.M * NP);
}

static int ipt_for(const Ctx& c) {
  const int NP = (c.N + 3) & ~3, items = (c.M / 2) * (NP / 4);
  return (items + kPT - 1) / kPT;
}

bool propagate_f32_ok(const Ctx& c) {
  return c.M % 2 == 0 && smem_propagate_f32(c) <= 200 * 1024 && ipt_for(c) <= 4;
}

cudaError_t prepare_propagate_f32() {
  const int lim = 200 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_propagate_f32<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_propagate_f32<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_propagate_f32<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_propagate_f32<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  return e;
}

// Phi' of every walker: reads c.phi (FP64) and c.Avhs32, writes out (FP64) and out32 (FP32,
// may be null).
cudaError_t launch_propagate_f32(const Ctx& c, double* out, float* out32, cudaStream_t s) {
  if (!propagate_f32_ok(c)) return cudaErrorInvalidValue;
  const size_t sm = smem_propagate_f32(c);
  const int order = c.opt.taylor_order;
#define AFQ_PROP(K)                                                                            \
  k_propagate_f32<K><<<c.Nw, kPT, sm, s>>>(c.phi, c.Avhs32, c.expK32, out, out32, c.M, c.N, c.Nw, \
                                           order)
  switch (ipt_for(c)) {
    case 1: AFQ_PROP(1); break;
    case 2: AFQ_PROP(2); break;
    case 3: AFQ_PROP(3); break;
    default: AFQ_PROP(4); break;
  }
#undef AFQ_PROP
  return cudaGetLastError();
}

}  // namespace afq
