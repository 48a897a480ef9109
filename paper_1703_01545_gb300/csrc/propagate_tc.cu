// Tensor-core one-step propagator of the split-precision path (Eq. 11 with the Taylor
// exponential), for M <= 64 orbitals and N <= 16 occupied columns:
//   Phi' = e^{-dt K/2} [ sum_{n<=order} A^n / n! ] e^{-dt K/2} Phi
// as eight dependent tcgen05 rounds per walker, each one MMA tile of M = 128 rows:
//   one-body   D = (E - I) X,  E = e^{-dt K/2}: rows 0..63 of the A operand hold E - I; the
//              result is X + D, so the identity part is added exactly in FP32;
//   Taylor     D = [A_re; A_im] [T_re T_im]^T (rows i and 64 + i, columns (re/im, b)), from
//              which T_n = (A_re T_re - A_im T_im + i (A_re T_im + A_im T_re)) / n.
// Operands are split BF16 (hi + lo, three MMAs per product, FP32 accumulation in TMEM), so a
// product carries ~2^-16 relative error: on the Taylor terms (whose size is ~|A| |T|) and on the
// small E - I part only.  Threads write the B operand (the current term) and A into shared
// memory in the 128-byte-swizzled K-major layout themselves; one elected thread issues the MMAs;
// the accumulator goes TMEM -> registers -> shared -> the threads that own the outputs.
// A persistent CTA (128 threads) loops over walkers; every mbarrier wait is bounded.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "tc_device.cuh"

namespace afq {
namespace {

using namespace tc;

constexpr uint64_t kPWaitNs = 2000000000ull;

// byte offset of bf16 element (r, k) in a K-major operand with 64-element (128-byte) rows and
// the 128-byte swizzle (16-byte chunk index XOR row mod 8), base 1024-byte aligned
__device__ __forceinline__ uint32_t sw128_off(int r, int k) {
  return (uint32_t)(r * 128 + ((((k >> 3) ^ r) & 7) << 4) + ((k & 7) << 1));
}

// split 8 FP32 values into bf16 hi / lo chunks (16 bytes each)
__device__ __forceinline__ void split8(const float (&x)[8], uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const __nv_bfloat16 a = __float2bfloat16_rn(x[2 * q]), b = __float2bfloat16_rn(x[2 * q + 1]);
    const __nv_bfloat16 c = __float2bfloat16_rn(x[2 * q] - __bfloat162float(a));
    const __nv_bfloat16 d = __float2bfloat16_rn(x[2 * q + 1] - __bfloat162float(b));
    h[q] = (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
    l[q] = (uint32_t)__bfloat16_as_ushort(c) | ((uint32_t)__bfloat16_as_ushort(d) << 16);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

template <int NPAD>
struct PLayout {
  static constexpr int NB = 2 * NPAD;            // B rows = MMA N
  static constexpr int E_HI = 0;                 // (E - I): 64 rows, followed by A_HI
  static constexpr int A_HI = 8192;              // [A_re; A_im]: 128 rows
  static constexpr int E_LO = A_HI + 16384;
  static constexpr int A_LO = E_LO + 8192;
  static constexpr int B_HI = A_LO + 16384;      // NB rows
  static constexpr int B_LO = B_HI + ((NB * 128 + 1023) / 1024) * 1024;
  static constexpr int S_OFF = B_LO + ((NB * 128 + 1023) / 1024) * 1024;
  static constexpr int SST = NB + 1;             // staging row stride (floats)
  static constexpr int BAR = S_OFF + 128 * SST * 4;
  static constexpr int SMEM_BYTES = ((BAR + 16 + 7) & ~7) + 1024;
};

template <int NPAD>
__global__ void __launch_bounds__(128, 3)
    k_propagate_tc(const double* __restrict__ phi_in, const float* __restrict__ Av,
                   const double* __restrict__ expK, double* __restrict__ phi_out,
                   float* __restrict__ phi_out32, int M, int N, int Nw, int order, int* err,
                   uint64_t wait_ns) {
  using Lay = PLayout<NPAD>;
  constexpr int NB = Lay::NB, TPR = 128 / NB, EPT = 64 / TPR, SST = Lay::SST;
  extern __shared__ uint8_t psm_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(psm_raw) + 1023) &
                                             ~uintptr_t(1023));
  float* S = reinterpret_cast<float*>(smem + Lay::S_OFF);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Lay::BAR);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
  __shared__ int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t base = smem_u32(smem), mbar = smem_u32(bar);
  // B-operand ownership: row n' = tid / TPR = (p, b), elements i0 .. i0 + EPT - 1
  const int nrow = tid / TPR, p = nrow / NPAD, b = nrow % NPAD, i0 = (tid % TPR) * EPT;
  const int64_t NM = (int64_t)N * M, plane = (int64_t)Nw * NM, MM = (int64_t)M * M;

  if (tid == 0) {
    mbar_init(mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_bad = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(32u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  // E - I (rows i < 64, K = j), zero outside M x M, once per CTA
  if (tid < 64) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      float x[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int j = 8 * c + q;
        x[q] = (tid < M && j < M) ? (float)(expK[(int64_t)tid * M + j] - (tid == j ? 1.0 : 0.0)) : 0.f;
      }
      uint4 h, l;
      split8(x, h, l);
      *reinterpret_cast<uint4*>(smem + Lay::E_HI + sw128_off(tid, 8 * c)) = h;
      *reinterpret_cast<uint4*>(smem + Lay::E_LO + sw128_off(tid, 8 * c)) = l;
    }
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = idesc_bf16<NB>();
  uint32_t round = 0;

  // one MMA round on the current B operand; afterwards the accumulator rows sit in S
  auto mma_round = [&](bool onebody) -> bool {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t ah = sw128_desc(base + (onebody ? Lay::E_HI : Lay::A_HI));
      const uint64_t al = sw128_desc(base + (onebody ? Lay::E_LO : Lay::A_LO));
      const uint64_t bh = sw128_desc(base + Lay::B_HI), bl = sw128_desc(base + Lay::B_LO);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t dk = (uint64_t)((kk * 32) >> 4);
        mma_bf16(tmem, ah + dk, bh + dk, idesc, kk != 0);
        mma_bf16(tmem, ah + dk, bl + dk, idesc, 1u);
        mma_bf16(tmem, al + dk, bh + dk, idesc, 1u);
      }
      mma_commit(mbar);
    }
    const bool ok = mbar_wait(mbar, round & 1, err, wait_ns);
    ++round;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) s_bad = 1;
    } else {
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
#pragma unroll
      for (int c = 0; c < NB; ++c) S[(warp * 32 + lane) * SST + c] = __uint_as_float(v[c]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    return s_bad == 0;
  };
  // the thread's part of a term -> B operand
  auto write_b = [&](const float (&x)[EPT]) {
#pragma unroll
    for (int c = 0; c < EPT / 8; ++c) {
      float y[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) y[q] = x[8 * c + q];
      uint4 h, l;
      split8(y, h, l);
      *reinterpret_cast<uint4*>(smem + Lay::B_HI + sw128_off(nrow, i0 + 8 * c)) = h;
      *reinterpret_cast<uint4*>(smem + Lay::B_LO + sw128_off(nrow, i0 + 8 * c)) = l;
    }
  };

  for (int w = blockIdx.x; w < Nw; w += gridDim.x) {
    // [A_re; A_im] rows r (A row i = r mod 64), 4 consecutive j per item: a warp reads two
    // whole rows per instruction (coalesced) and stores 8-byte halves of swizzled chunks
    for (int e = tid; e < 128 * 16; e += 128) {
      const int r = e >> 4, j0 = (e & 15) * 4, i = r & 63;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i < M && j0 < M)
        v = __ldg(reinterpret_cast<const float4*>(Av + (r < 64 ? 0 : (int64_t)Nw * MM) +
                                                  (int64_t)w * MM + (int64_t)i * M + j0));
      const float x[4] = {v.x, v.y, v.z, v.w};
      uint32_t h[2], l[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const __nv_bfloat16 a0 = __float2bfloat16_rn(x[2 * q]), a1 = __float2bfloat16_rn(x[2 * q + 1]);
        const __nv_bfloat16 l0 = __float2bfloat16_rn(x[2 * q] - __bfloat162float(a0));
        const __nv_bfloat16 l1 = __float2bfloat16_rn(x[2 * q + 1] - __bfloat162float(a1));
        h[q] = (uint32_t)__bfloat16_as_ushort(a0) | ((uint32_t)__bfloat16_as_ushort(a1) << 16);
        l[q] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
      }
      *reinterpret_cast<uint2*>(smem + Lay::A_HI + sw128_off(r, j0)) = make_uint2(h[0], h[1]);
      *reinterpret_cast<uint2*>(smem + Lay::A_LO + sw128_off(r, j0)) = make_uint2(l[0], l[1]);
    }
    // the walker, coalesced into the staging buffer as [p][b][i] (64 floats per column)
    for (int e = tid; e < 2 * NPAD * 64; e += 128) {
      const int pp = e / (NPAD * 64), bb = (e / 64) % NPAD, i = e % 64;
      S[e] = (bb < N && i < M) ? (float)phi_in[(int64_t)pp * plane + ((int64_t)w * N + bb) * M + i] : 0.f;
    }
    __syncthreads();
    float X[EPT], Ssum[EPT], T[EPT];
#pragma unroll
    for (int q = 0; q < EPT; ++q) X[q] = S[nrow * 64 + i0 + q];
    // Phi1 = Phi + (E - I) Phi
    write_b(X);
    if (!mma_round(true)) break;
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      T[q] = X[q] + S[(i0 + q) * SST + p * NPAD + b];
      Ssum[q] = T[q];
    }
    // Taylor terms
    for (int n = 1; n <= order; ++n) {
      __syncthreads();   // every thread has read S before the next round overwrites it
      write_b(T);
      if (!mma_round(false)) break;
      const float inv = 1.f / (float)n;
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const int i = i0 + q;
        const float rr = S[i * SST + b], ri = S[i * SST + NPAD + b];               // A_re T_re, A_re T_im
        const float ir = S[(64 + i) * SST + b], ii = S[(64 + i) * SST + NPAD + b]; // A_im T_re, A_im T_im
        T[q] = (p == 0 ? rr - ii : ri + ir) * inv;
        Ssum[q] += T[q];
      }
    }
    if (s_bad) break;
    // Phi' = Phi2 + (E - I) Phi2
    __syncthreads();
    write_b(Ssum);
    if (!mma_round(true)) break;
#pragma unroll
    for (int q = 0; q < EPT; ++q) X[q] = Ssum[q] + S[(i0 + q) * SST + p * NPAD + b];
    __syncthreads();   // every thread has read the accumulator rows from S
#pragma unroll
    for (int q = 0; q < EPT; ++q) S[nrow * 64 + i0 + q] = X[q];
    __syncthreads();
    for (int e = tid; e < 2 * NPAD * 64; e += 128) {   // coalesced write of the walker
      const int pp = e / (NPAD * 64), bb = (e / 64) % NPAD, i = e % 64;
      if (bb < N && i < M) {
        const int64_t g = (int64_t)pp * plane + ((int64_t)w * N + bb) * M + i;
        phi_out[g] = (double)S[e];
        if (phi_out32) phi_out32[g] = S[e];
      }
    }
    __syncthreads();   // S and the operands are reused by the next walker
  }
  // after an expired wait the MMAs of that round may still be in flight: wait (bounded) for
  // their commit before the accumulator is freed
  if (s_bad && tid == 0) mbar_wait(mbar, (round - 1) & 1, err, wait_ns);
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32u)
                 : "memory");
}

}  // namespace

bool propagate_tc_ok(const Ctx& c) {
  return c.M <= 64 && c.M % 4 == 0 && c.N <= 16 && c.N >= 1;
}

cudaError_t prepare_propagate_tc() {
  cudaError_t e = cudaFuncSetAttribute(k_propagate_tc<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       PLayout<8>::SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_propagate_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             PLayout<16>::SMEM_BYTES);
  return e;
}

// Phi' of every walker from c.phi and c.Avhs32: out (FP64), out32 (FP32, may be null).
cudaError_t launch_propagate_tc(const Ctx& c, double* out, float* out32, cudaStream_t s) {
  if (!propagate_tc_ok(c)) return cudaErrorInvalidValue;
  const int grid = std::min(c.Nw, 152 * 3);
  if (c.N <= 8)
    k_propagate_tc<8><<<grid, 128, PLayout<8>::SMEM_BYTES, s>>>(c.phi, c.Avhs32, c.expK, out, out32, c.M,
                                                               c.N, c.Nw, c.opt.taylor_order,
                                                               c.d_tc_err, kPWaitNs);
  else
    k_propagate_tc<16><<<grid, 128, PLayout<16>::SMEM_BYTES, s>>>(c.phi, c.Avhs32, c.expK, out, out32,
                                                                 c.M, c.N, c.Nw, c.opt.taylor_order,
                                                                 c.d_tc_err, kPWaitNs);
  return cudaGetLastError();
}

}  // namespace afq
