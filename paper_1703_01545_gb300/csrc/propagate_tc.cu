// Tensor-core one-step propagator of the split-precision path (Eq. 11 with the Taylor
// exponential), for M <= 64 orbitals and N <= 16 occupied columns:
//   Phi' = e^{-dt K/2} [ sum_{n<=order} A^n / n! ] e^{-dt K/2} Phi
// as eight dependent tcgen05 rounds per walker, each one MMA tile of M = 128 rows.  Row r of
// every accumulator is the real (r < 64) or imaginary (r >= 64) part of orbital row i = r % 64,
// with the occupied column b along N, so thread r owns the same numbers in every round and no
// accumulator passes through shared memory:
//   one-body   D = [E - I; E - I] [X_re; X_im]^T  (N = 32: thread r takes columns 16 p .. 16 p + 15),
//              E = e^{-dt K/2}; the result is X + D, so the identity part is added exactly in FP32.
//              The constant operand [E - I; E - I] lives in tensor memory (written once per CTA
//              by the thread that owns each row), which keeps shared memory at ~57 KB per CTA;
//   Taylor     D = [A_re  -A_im; A_im  A_re] [T_re  T_im]^T  (K = 128, N = 16), which is
//              [Re(A T); Im(A T)]; T_n = D / n.
// The K = 128 operand is stored once as the 192 rows [-A_im; A_re; A_im]: its first K block
// (K = j of T_re) is rows 64..191, the second (K = j of T_im) rows 0..127.  Operands are split
// BF16 (hi + lo, three MMAs per product, FP32 accumulation in TMEM), so a product carries
// ~2^-16 relative error: on the Taylor terms (whose size is ~|A| |T|) and on the small E - I
// part only.  Thread r writes its column K = i of the B operand (16 rows b, 2-byte stores into
// the 128-byte-swizzled K-major layout); one elected thread issues the MMAs.  A persistent CTA
// (128 threads, three per SM) loops over walkers, prefetching the next walker's inputs to L2;
// every mbarrier wait is bounded.
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

struct PLayout {
  static constexpr int A_HI = 0;                 // [-A_im; A_re; A_im]: 192 rows, K = j
  static constexpr int A_LO = A_HI + 24576;
  static constexpr int B_HI = A_LO + 24576;      // rows b of the real part, then of the imaginary
  static constexpr int B_LO = B_HI + 4096;       // part (16 + 16 rows, K = j)
  static constexpr int BAR = B_LO + 4096;
  static constexpr int SMEM_BYTES = BAR + 16 + 1024;
  // tensor memory columns: accumulator, then [E - I; E - I] as the A operand (K = 64, two
  // bf16 per column): hi and lo
  static constexpr uint32_t T_COLS = 128, T_EHI = 32, T_ELO = 64;
};

__global__ void __launch_bounds__(128, 3)
    k_propagate_tc(const double* phi_in, const float* __restrict__ Av,
                   const uint32_t* __restrict__ emI_pk, double* phi_out,
                   float* __restrict__ phi_out32, const int* __restrict__ alive, int M, int N,
                   int Nw, int order, int* err, uint64_t wait_ns) {
  using Lay = PLayout;
  extern __shared__ uint8_t psm_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(psm_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Lay::BAR);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t base = smem_u32(smem), mbar = smem_u32(bar);
  // accumulator row tid: part p (0 real, 1 imaginary) of orbital row i
  const int p = tid >> 6, i = tid & 63;
  const int64_t NM = (int64_t)N * M, plane = (int64_t)Nw * NM, MM = (int64_t)M * M;

  if (tid == 0) {
    mbar_init(mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(Lay::T_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);   // this warp's TMEM lanes
  // [E - I; E - I] into tensor memory, once per CTA: lane tid holds row i (the split-bf16 words
  // packed at setup: 32 hi words, then 32 lo words)
#pragma unroll 1
  for (int cc = 0; cc < 4; ++cc) {
    const uint4* src = reinterpret_cast<const uint4*>(emI_pk + i * 64 + 8 * cc);
    const uint4 h0 = __ldg(src), h1 = __ldg(src + 1), l0 = __ldg(src + 8), l1 = __ldg(src + 9);
    const uint32_t vh[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
    const uint32_t vl[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
    tmem_st8(tl + Lay::T_EHI + 8 * cc, vh);
    tmem_st8(tl + Lay::T_ELO + 8 * cc, vl);
  }
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  const uint32_t id16 = idesc_bf16<16>(), id32 = idesc_bf16<32>();
  uint32_t phase = 0;
  bool failed = false;
  // B operand: this thread's column K = i in row b of its part p (rows b + 8 lie 1024 bytes on)
  uint32_t boff[8];
#pragma unroll
  for (int b = 0; b < 8; ++b) boff[b] = Lay::B_HI + p * 2048 + sw128_off(b, i);
  auto write_b = [&](const float (&x)[16]) {
#pragma unroll
    for (int b = 0; b < 16; ++b) {
      const __nv_bfloat16 h = __float2bfloat16_rn(x[b]);
      const __nv_bfloat16 l = __float2bfloat16_rn(x[b] - __bfloat162float(h));
      uint8_t* q = smem + boff[b & 7] + (b >> 3) * 1024;
      *reinterpret_cast<uint16_t*>(q) = __bfloat16_as_ushort(h);
      *reinterpret_cast<uint16_t*>(q + (Lay::B_LO - Lay::B_HI)) = __bfloat16_as_ushort(l);
    }
  };
  // one MMA round on the B operand just written; false when a wait expired (in any thread)
  auto mma_round = [&](bool onebody) -> bool {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    if (__syncthreads_or(failed ? 1 : 0)) return false;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t bh = sw128_desc(base + Lay::B_HI), bl = sw128_desc(base + Lay::B_LO);
      if (onebody) {
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t dk = (uint64_t)(2 * kk);          // 16 bf16 = 32 bytes along K
          const uint32_t eh = tmem + Lay::T_EHI + 8 * kk, el = tmem + Lay::T_ELO + 8 * kk;
          mma_bf16_ta(tmem, eh, bh + dk, id32, kk != 0);
          mma_bf16_ta(tmem, eh, bl + dk, id32, 1u);
          mma_bf16_ta(tmem, el, bh + dk, id32, 1u);
        }
      } else {
#pragma unroll
        for (int blk = 0; blk < 2; ++blk) {
          // K block 0 (T_re): operand rows 64..191 = [A_re; A_im]; K block 1 (T_im): rows
          // 0..127 = [-A_im; A_re]
          const uint32_t ao = blk ? 0u : 8192u, bo = blk ? 2048u : 0u;
          const uint64_t ah = sw128_desc(base + Lay::A_HI + ao), al = sw128_desc(base + Lay::A_LO + ao);
          const uint64_t bbh = bh + (bo >> 4), bbl = bl + (bo >> 4);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t dk = (uint64_t)(2 * kk);
            mma_bf16(tmem, ah + dk, bbh + dk, id16, (blk | kk) != 0);
            mma_bf16(tmem, ah + dk, bbl + dk, id16, 1u);
            mma_bf16(tmem, al + dk, bbh + dk, id16, 1u);
          }
        }
      }
      mma_commit(mbar);
    }
    if (!mbar_wait(mbar, phase & 1, err, wait_ns)) failed = true;
    ++phase;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return true;
  };

  for (int w = blockIdx.x; w < Nw; w += gridDim.x) {
    // in place (phi_out == phi_in), dead walkers keep their Phi: each walker's inputs are read
    // in full before any of its outputs is written
    if (alive && !alive[w]) continue;
    // the next walker's A planes and Phi towards L2 while this one is propagated
    if (tid == 0 && w + (int)gridDim.x < Nw) {
      const int wn = w + gridDim.x;
      const uint32_t abytes = (uint32_t)(MM * 4), pbytes = (uint32_t)(NM * 8);
      const float* a0 = Av + (int64_t)wn * MM;
      const double* f0 = phi_in + (int64_t)wn * NM;
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a0), "r"(abytes) : "memory");
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a0 + (int64_t)Nw * MM), "r"(abytes) : "memory");
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(f0), "r"(pbytes) : "memory");
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(f0 + plane), "r"(pbytes) : "memory");
    }
    // [-A_im; A_re; A_im]: item q of this thread is A row (q % 8) * 8 + tid / 16 of the real
    // (q < 8) or imaginary plane, 4 consecutive j; a warp reads two whole rows per load
    {
      float4 av[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int ii = ((q & 7) << 3) + (tid >> 4), j0 = (tid & 15) * 4;
        av[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ii < M && j0 < M)
          av[q] = __ldg(reinterpret_cast<const float4*>(Av + (q < 8 ? 0 : (int64_t)Nw * MM) +
                                                        (int64_t)w * MM + (int64_t)ii * M + j0));
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int ii = ((q & 7) << 3) + (tid >> 4), j0 = (tid & 15) * 4;
        const float x[4] = {av[q].x, av[q].y, av[q].z, av[q].w};
        uint32_t h[2], l[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const __nv_bfloat16 a0 = __float2bfloat16_rn(x[2 * e]), a1 = __float2bfloat16_rn(x[2 * e + 1]);
          const __nv_bfloat16 l0 = __float2bfloat16_rn(x[2 * e] - __bfloat162float(a0));
          const __nv_bfloat16 l1 = __float2bfloat16_rn(x[2 * e + 1] - __bfloat162float(a1));
          h[e] = (uint32_t)__bfloat16_as_ushort(a0) | ((uint32_t)__bfloat16_as_ushort(a1) << 16);
          l[e] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
        }
        // real part -> row 64 + ii; imaginary part -> row 128 + ii and, negated, row ii
        const uint32_t o = sw128_off((q < 8 ? 64 : 128) + ii, j0);
        *reinterpret_cast<uint2*>(smem + Lay::A_HI + o) = make_uint2(h[0], h[1]);
        *reinterpret_cast<uint2*>(smem + Lay::A_LO + o) = make_uint2(l[0], l[1]);
        if (q >= 8) {
          const uint32_t on = sw128_off(ii, j0), sg = 0x80008000u;
          *reinterpret_cast<uint2*>(smem + Lay::A_HI + on) = make_uint2(h[0] ^ sg, h[1] ^ sg);
          *reinterpret_cast<uint2*>(smem + Lay::A_LO + on) = make_uint2(l[0] ^ sg, l[1] ^ sg);
        }
      }
    }
    // this thread's row of the walker: part p of orbital i, columns b (coalesced over i)
    float X[16], T[16], Ssum[16];
    uint32_t v[16];
#pragma unroll
    for (int b = 0; b < 16; ++b)
      X[b] = (b < N && i < M) ? (float)phi_in[(int64_t)p * plane + ((int64_t)w * N + b) * M + i] : 0.f;
    // Phi1 = Phi + (E - I) Phi
    write_b(X);
    if (!mma_round(true)) break;
    tmem_ld16(tl + (p ? 16u : 0u), v);
#pragma unroll
    for (int b = 0; b < 16; ++b) {
      T[b] = X[b] + __uint_as_float(v[b]);
      Ssum[b] = T[b];
    }
    // Taylor terms T_n = A T_{n-1} / n
    bool ok = true;
    for (int n = 1; n <= order && ok; ++n) {
      write_b(T);
      ok = mma_round(false);
      if (ok) {
        tmem_ld16(tl, v);
        const float inv = 1.f / (float)n;
#pragma unroll
        for (int b = 0; b < 16; ++b) {
          T[b] = __uint_as_float(v[b]) * inv;
          Ssum[b] += T[b];
        }
      }
    }
    if (!ok) break;
    // Phi' = Phi2 + (E - I) Phi2
    write_b(Ssum);
    if (!mma_round(true)) break;
    tmem_ld16(tl + (p ? 16u : 0u), v);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    if (__syncthreads_or(failed ? 1 : 0)) break;
    if (i < M)
#pragma unroll
      for (int b = 0; b < 16; ++b)
        if (b < N) {
          const float y = Ssum[b] + __uint_as_float(v[b]);
          const int64_t g = (int64_t)p * plane + ((int64_t)w * N + b) * M + i;
          phi_out[g] = (double)y;
          if (phi_out32) phi_out32[g] = y;
        }
  }
  // after an expired wait the MMAs of that round may still be in flight: wait (bounded) for
  // their commit before the accumulator is freed
  if (__syncthreads_or(failed ? 1 : 0) && tid == 0 && phase > 0) mbar_wait(mbar, (phase - 1) & 1, err, wait_ns);
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Lay::T_COLS)
                 : "memory");
}

// emI_pk[r][c]: row r of e^{-dt K/2} - I (formed in FP64, rounded to FP32, zero outside M x M)
// split into bf16 hi + lo; words 0..31 hold hi pairs (k = 2c, 2c + 1), words 32..63 lo pairs
__global__ void k_pack_emI(const double* __restrict__ expK, int M, uint32_t* __restrict__ out) {
  const int r = blockIdx.x, c = threadIdx.x;   // 64 x 32
  float x[2];
  for (int q = 0; q < 2; ++q) {
    const int j = 2 * c + q;
    x[q] = (r < M && j < M) ? (float)(expK[(int64_t)r * M + j] - (r == j ? 1.0 : 0.0)) : 0.f;
  }
  uint16_t h[2], l[2];
  for (int q = 0; q < 2; ++q) {
    const __nv_bfloat16 hb = __float2bfloat16_rn(x[q]);
    h[q] = __bfloat16_as_ushort(hb);
    l[q] = __bfloat16_as_ushort(__float2bfloat16_rn(x[q] - __bfloat162float(hb)));
  }
  out[r * 64 + c] = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
  out[r * 64 + 32 + c] = (uint32_t)l[0] | ((uint32_t)l[1] << 16);
}

}  // namespace

cudaError_t pack_propagate_tc(const Ctx& c, uint32_t* emI_pk, cudaStream_t s) {
  k_pack_emI<<<64, 32, 0, s>>>(c.expK, c.M, emI_pk);
  return cudaGetLastError();
}

bool propagate_tc_ok(const Ctx& c) {
  return c.M <= 64 && c.M % 4 == 0 && c.N <= 16 && c.N >= 1;
}

cudaError_t prepare_propagate_tc() {
  return cudaFuncSetAttribute(k_propagate_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              PLayout::SMEM_BYTES);
}

// Phi' of every walker from c.phi and c.Avhs32: out (FP64), out32 (FP32, may be null).  With
// out == c.phi the live walkers are propagated in place and the dead ones left as they are.
cudaError_t launch_propagate_tc(const Ctx& c, double* out, float* out32, cudaStream_t s) {
  if (!propagate_tc_ok(c)) return cudaErrorInvalidValue;
  const int grid = std::min(c.Nw, 152 * 3);
  if (!c.emI_pk) return cudaErrorInvalidValue;
  k_propagate_tc<<<grid, 128, PLayout::SMEM_BYTES, s>>>(c.phi, c.Avhs32, c.emI_pk, out, out32,
                                                        out == c.phi ? c.alive : nullptr, c.M, c.N,
                                                        c.Nw, c.opt.taylor_order, c.d_tc_err, kPWaitNs);
  return cudaGetLastError();
}

}  // namespace afq
