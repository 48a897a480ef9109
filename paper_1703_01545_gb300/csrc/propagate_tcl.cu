// Tensor-core one-step propagator of the split-precision path for M <= 256 orbitals and
// N <= 32 occupied columns (Eq. 11 with the Taylor exponential):
//   Phi' = e^{-dt K/2} [ sum_{n<=order} A^n / n! ] e^{-dt K/2} Phi.
//
// Each product is one accumulation per 128-row tile of orbitals i (one tile for M <= 128, two
// up to 256) with the occupied columns of the term along the MMA's N dimension, real parts
// then imaginary parts (N = 2 Np, Np = N rounded up to 8):
//   Taylor    D = A_re [T_re | T_im] + A_im [-T_im | T_re] = [Re(A T) | Im(A T)]
//   one-body  D = (E - I) [X_re | X_im],  E = e^{-dt K/2}, X + D formed in FP32
// Both B operands are windows of one buffer of 3 Np rows [-T_im; T_re; T_im] (K = orbital j):
// rows Np..3Np serve A_re and E - I, rows 0..2Np serve A_im.
//
// A is not held in shared memory: its split-BF16 tiles (128 rows x 64 K, hi and lo, written in
// that form by the V_HS contraction) stream through a TMA ring for every round, so the ring
// and the term operand fit two CTAs per SM at M = 128.  A hi tile is consumed by two MMAs per
// 16-wide K step (hi * T_hi, hi * T_lo), a lo tile by one (lo * T_hi): the three split
// products, accumulated in FP32 in tensor memory.  The running sum S of the series lives in
// tensor memory beside the accumulator, so the epilogue threads hold no more than 16 columns
// at a time.
//
// Roles (persistent CTA over walkers, 192 threads):
//   warp 0 / lane 0  TMA producer: the tiles of every round of every walker, in order
//   warp 1 / lane 0  MMA issuer: per round, waits for the term operand, consumes the tiles,
//                    commits "D full"
//   warps 2..5       epilogue: thread r owns orbital row i = 128 t + r of every tile t (TMEM
//                    lane r); reads D and S, forms the next term, writes it into the operand
//                    (split BF16, 128-byte swizzle), arrives on "B ready"
// Every wait is bounded by %globaltimer; on expiry the kernel sets *err and a shared abort
// flag, every role leaves its loop, in-flight TMA loads and MMAs are waited for (bounded) and
// the tensor memory is freed.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "tc_device.cuh"

namespace afq {
namespace {

using namespace tc;

constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int kTile = 128 * 64 * 2;       // one 128-row x 64-K bf16 tile, 128-byte swizzle
constexpr int kMaxStages = 12;

__device__ __forceinline__ uint32_t sw128_off(int r, int k) {
  return (uint32_t)(r * 128 + ((((k >> 3) ^ r) & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint32_t idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x,
                                            int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}

// L2 prefetch hint over the 16-byte-aligned interior of [p, p + bytes) (the bulk prefetch needs a
// 16-byte-aligned address and size)
__device__ __forceinline__ void prefetch_l2(const void* p, uint64_t bytes) {
  const uint64_t a = reinterpret_cast<uint64_t>(p);
  const uint64_t lo = (a + 15) & ~uint64_t(15), hi = (a + bytes) & ~uint64_t(15);
  if (hi > lo)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((uint32_t)(hi - lo))
                 : "memory");
}

// Static shape of one launch (host-computed).
struct TclShape {
  const __nv_bfloat16 *ahi, *alo;   // V_HS split planes [2][Nw][M][Mp] (L2 prefetch of the next walker)
  int Mp;                // elements per orbital row of the split planes
  int M, N, Np, n2;      // orbitals, occupied columns, N rounded up to 8, MMA N = 2 Np
  int MT, KB;            // 128-row tiles of orbitals, 64-wide K blocks
  int nst;               // ring stages
  int resident;          // 1: A of a walker held in shared memory for all its Taylor rounds
  int ares_off;          // resident A region: 4 KB tiles (A_re hi, lo, A_im hi, lo per K block)
  int bkb;               // bytes of one K block of the term operand (3 Np rows x 128 bytes)
  int dcol;              // TMEM column stride between tiles (D and S regions)
  uint32_t tcols;        // TMEM columns allocated
  int order, Nw;
  int ring_off, bhi_off, blo_off, bar_off, smem_bytes;
};

// Round q of a walker: 0 and order + 1 are the one-body products, 1..order the Taylor terms.
// Tiles of a round, in order: for each row tile t and K block kb: E hi, E lo (one-body) or
// A_re hi, A_re lo, A_im hi, A_im lo (Taylor).

template <int EPI>
__global__ void __launch_bounds__(64 + 32 * EPI, EPI == 4 ? 2 : 1)
    k_propagate_tcl(const __grid_constant__ CUtensorMap tmAhi, const __grid_constant__ CUtensorMap tmAlo,
                    const __grid_constant__ CUtensorMap tmEhi, const __grid_constant__ CUtensorMap tmElo,
                    const TclShape sh, const double* phi_in, double* phi_out,
                    float* __restrict__ phi_out32, const int* __restrict__ alive, int* err,
                    uint64_t wait_ns) {
  extern __shared__ uint8_t tsm_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tsm_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + sh.bar_off);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + kMaxStages);
  const uint32_t dfull = smem_u32(bars + 2 * kMaxStages), bready = smem_u32(bars + 2 * kMaxStages + 1);
  const uint32_t done = smem_u32(bars + 2 * kMaxStages + 2);
  const uint32_t afull = smem_u32(bars + 2 * kMaxStages + 3), aempty = smem_u32(bars + 2 * kMaxStages + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kMaxStages + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rounds = sh.order + 2;
  const int64_t NM = (int64_t)sh.N * sh.M, plane = (int64_t)sh.Nw * NM;

  if (threadIdx.x == 0) {
    for (int q = 0; q < sh.nst; ++q) {
      mbar_init(full0 + 8 * q, 1);
      mbar_init(empty0 + 8 * q, 1);
    }
    mbar_init(dfull, 1);
    mbar_init(bready, 32 * EPI);
    mbar_init(done, 1);
    mbar_init(afull, 1);
    mbar_init(aempty, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // the term operand starts at zero: padded rows and K beyond M stay zero throughout
  for (int e = threadIdx.x; e < 2 * sh.KB * sh.bkb / 16; e += blockDim.x)
    reinterpret_cast<uint4*>(smem + sh.bhi_off)[e] = make_uint4(0u, 0u, 0u, 0u);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor core
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(sh.tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  auto fail = [&]() { *abort_flag = 1; };

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer: the same walker and tile order the MMA issuer consumes ----
      int g = 0, aw = 0;
      bool ok = true;
      const uint64_t abytes = (uint64_t)sh.M * sh.Mp * 2;   // one plane of A, hi or lo
      const uint64_t pbytes = (uint64_t)NM * 8;             // one plane of Phi
      for (int w = blockIdx.x; w < sh.Nw && ok; w += gridDim.x) {
        if (alive && !alive[w]) continue;
        // the next walker's A planes and Phi towards L2 while this one is propagated
        const int wn = w + gridDim.x;
        if (wn < sh.Nw) {
          for (int z = 0; z < 2; ++z) {
            const int64_t ao = ((int64_t)z * sh.Nw + wn) * sh.M * sh.Mp;
            prefetch_l2(sh.ahi + ao, abytes);
            prefetch_l2(sh.alo + ao, abytes);
            prefetch_l2(phi_in + z * plane + (int64_t)wn * NM, pbytes);
          }
        }
        for (int q = 0; q < rounds && ok; ++q) {
          const bool taylor = q >= 1 && q <= sh.order;
          if (sh.resident && taylor) {
            if (q == 1) {
              // this walker's A into the resident region once the previous walker's last
              // Taylor round has read it (aempty), all tiles on one barrier
              if (aw > 0 && !mbar_wait(aempty, (aw - 1) & 1, err, wait_ns)) {
                fail();
                ok = false;
                break;
              }
              mbar_expect_tx(afull, 4 * sh.KB * kTile);
              for (int kb = 0; kb < sh.KB; ++kb)
                for (int u = 0; u < 4; ++u)
                  tma_load_3d(smem_u32(smem + sh.ares_off + (kb * 4 + u) * kTile),
                              (u & 1) ? &tmAlo : &tmAhi, afull, kb * 64, 0, (u >> 1) * sh.Nw + w);
              ++aw;
            }
            continue;
          }
          for (int t = 0; t < sh.MT && ok; ++t)
            for (int kb = 0; kb < sh.KB && ok; ++kb)
              for (int u = 0; u < (taylor ? 4 : 2); ++u, ++g) {
                const int st = g % sh.nst, use = g / sh.nst;
                if (*abort_flag) { ok = false; break; }
                if (g >= sh.nst && !mbar_wait(empty0 + 8 * st, (use - 1) & 1, err, wait_ns)) {
                  fail();
                  ok = false;
                  break;
                }
                const uint32_t dst = smem_u32(smem + sh.ring_off + st * kTile);
                const uint32_t fb = full0 + 8 * st;
                mbar_expect_tx(fb, kTile);
                if (taylor) {
                  // u: 0 A_re hi, 1 A_re lo, 2 A_im hi, 3 A_im lo; z = (plane, walker)
                  const int z = (u >> 1) * sh.Nw + w;
                  tma_load_3d(dst, (u & 1) ? &tmAlo : &tmAhi, fb, kb * 64, t * 128, z);
                } else {
                  tma_load_2d(dst, (u & 1) ? &tmElo : &tmEhi, fb, kb * 64, t * 128);
                }
              }
        }
      }
      // every issued tile must have landed before the CTA may exit
      for (int q = (g > sh.nst ? g - sh.nst : 0); q < g; ++q)
        mbar_wait(full0 + 8 * (q % sh.nst), (q / sh.nst) & 1, err, wait_ns);
      if (aw > 0) mbar_wait(afull, (aw - 1) & 1, err, wait_ns);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer ----
      const uint32_t idesc = idesc_n(sh.n2);
      const uint32_t bhi = smem_u32(smem + sh.bhi_off), blo = smem_u32(smem + sh.blo_off);
      int g = 0, rq = 0, aw = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < sh.Nw && ok; w += gridDim.x) {
        if (alive && !alive[w]) continue;
        for (int q = 0; q < rounds && ok; ++q, ++rq) {
          const bool taylor = q >= 1 && q <= sh.order;
          if (*abort_flag || !mbar_wait(bready, rq & 1, err, wait_ns)) { fail(); ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          if (sh.resident && taylor) {
            // A resident in shared memory: one tile row (MT = 1), the K blocks' four tiles
            if (q == 1) {
              if (!mbar_wait(afull, aw & 1, err, wait_ns)) { fail(); ok = false; break; }
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
              ++aw;
            }
            bool first = true;
            for (int kb = 0; kb < sh.KB; ++kb) {
              const int nks = min(4, (sh.M - 64 * kb + 15) / 16);
              for (int u = 0; u < 4; ++u) {
                const uint64_t a = sw128_desc(smem_u32(smem + sh.ares_off + (kb * 4 + u) * kTile));
                const uint32_t roff = (uint32_t)(kb * sh.bkb + (u >= 2 ? 0 : sh.Np * 128));
                const uint64_t bh = sw128_desc(bhi + roff), bl = sw128_desc(blo + roff);
                const bool hi = (u & 1) == 0;
                for (int ks = 0; ks < nks; ++ks) {
                  const uint64_t dk = (uint64_t)(2 * ks);
                  mma_bf16(tmem, a + dk, bh + dk, idesc, first ? 0u : 1u);
                  first = false;
                  if (hi) mma_bf16(tmem, a + dk, bl + dk, idesc, 1u);
                }
              }
            }
            if (q == sh.order) mma_commit(aempty);   // the region is free once these complete
            mma_commit(dfull);
            continue;
          }
          for (int t = 0; t < sh.MT && ok; ++t) {
            const uint32_t d = tmem + (uint32_t)(t * sh.dcol);
            bool first = true;
            for (int kb = 0; kb < sh.KB && ok; ++kb) {
              const int nks = min(4, (sh.M - 64 * kb + 15) / 16);   // K steps holding orbitals
              for (int u = 0; u < (taylor ? 4 : 2); ++u, ++g) {
                const int st = g % sh.nst, use = g / sh.nst;
                if (*abort_flag || !mbar_wait(full0 + 8 * st, use & 1, err, wait_ns)) {
                  fail();
                  ok = false;
                  break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t a = sw128_desc(smem_u32(smem + sh.ring_off + st * kTile));
                // A_im (u >= 2) takes rows 0..2Np of the term operand, A_re and E - I rows Np..3Np
                const uint32_t roff = (uint32_t)(kb * sh.bkb + ((taylor && u >= 2) ? 0 : sh.Np * 128));
                const uint64_t bh = sw128_desc(bhi + roff), bl = sw128_desc(blo + roff);
                const bool hi = (u & 1) == 0;
                for (int ks = 0; ks < nks; ++ks) {
                  const uint64_t dk = (uint64_t)(2 * ks);     // 16 bf16 = 32 bytes along K
                  mma_bf16(d, a + dk, bh + dk, idesc, first ? 0u : 1u);
                  first = false;
                  if (hi) mma_bf16(d, a + dk, bl + dk, idesc, 1u);
                }
                mma_commit(empty0 + 8 * st);
              }
            }
          }
          if (ok) mma_commit(dfull);
        }
      }
      mma_commit(done);   // arrives once every issued MMA has completed
    }
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31; with 8 epilogue warps two
    // share each lane quadrant and take alternate 16-column chunks ----
    const int r = 32 * (warp & 3) + lane;
    const int half = EPI == 8 ? (warp - 2) >> 2 : 0, cstep = EPI == 8 ? 32 : 16;
    const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
    uint8_t* bh8 = smem + sh.bhi_off;
    uint8_t* bl8 = smem + sh.blo_off;
    const uint32_t sreg = (uint32_t)(sh.MT * sh.dcol);   // S region after the D columns
    // term operand entry (row R, K = i): split BF16 into both halves
    auto put = [&](int R, int i, float x) {
      const uint32_t o = (uint32_t)((i >> 6) * sh.bkb) + sw128_off(R, i & 63);
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      *reinterpret_cast<__nv_bfloat16*>(bh8 + o) = h;
      *reinterpret_cast<__nv_bfloat16*>(bl8 + o) = __float2bfloat16_rn(x - __bfloat162float(h));
    };
    // column c of a tile: real part of column b = c (c < Np) or imaginary part of b = c - Np
    auto put_term = [&](int i, int c, float x, bool neg_copy) {
      if (c < sh.Np) {
        put(sh.Np + c, i, x);
      } else {
        put(sh.Np + c, i, x);                 // rows 2Np..3Np: T_im
        if (neg_copy) put(c - sh.Np, i, -x);  // rows 0..Np: -T_im
      }
    };
    int rq = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < sh.Nw && ok; w += gridDim.x) {
      if (alive && !alive[w]) continue;
      // S = X (this walker's columns) and the operand [X_re; X_im] for the first one-body round
      for (int t = 0; t < sh.MT; ++t) {
        const int i = 128 * t + r;
        const bool in_b = i < 64 * sh.KB;
        for (int c0 = 16 * half; c0 < sh.n2; c0 += cstep) {
          // the chunk's 16 loads first, all in flight together, then the operand stores
          double xv[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int c = c0 + e, b = c < sh.Np ? c : c - sh.Np;
            xv[e] = (i < sh.M && b < sh.N)
                        ? phi_in[(c < sh.Np ? 0 : plane) + ((int64_t)w * sh.N + b) * sh.M + i]
                        : 0.0;
          }
          uint32_t v[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const float x = (float)xv[e];
            v[e] = __float_as_uint(x);
            if (in_b) put_term(i, c0 + e, x, false);
          }
          tmem_st16(tmem + lanes + sreg + (uint32_t)(t * sh.dcol + c0), v);
        }
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(bready);
      for (int q = 0; q < rounds && ok; ++q, ++rq) {
        const bool last = q == rounds - 1;
        const bool okw = !*abort_flag && mbar_wait(dfull, rq & 1, err, wait_ns);
        if (!__all_sync(0xffffffffu, okw)) { fail(); ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const float inv = (q >= 1 && q <= sh.order) ? 1.f / (float)q : 1.f;
        for (int t = 0; t < sh.MT; ++t) {
          const int i = 128 * t + r;
          const bool in_b = i < 64 * sh.KB;
          for (int c0 = 16 * half; c0 < sh.n2; c0 += cstep) {
            uint32_t dv[16], sv[16];
            tmem_ld16(tmem + lanes + (uint32_t)(t * sh.dcol + c0), dv);
            tmem_ld16(tmem + lanes + sreg + (uint32_t)(t * sh.dcol + c0), sv);
            if (q == 0) {
              // T_0 = X + (E - I) X: S = T_0, operand = T_0
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                const float x = __uint_as_float(sv[e]) + __uint_as_float(dv[e]);
                sv[e] = __float_as_uint(x);
                if (in_b) put_term(i, c0 + e, x, true);
              }
              tmem_st16(tmem + lanes + sreg + (uint32_t)(t * sh.dcol + c0), sv);
            } else if (!last) {
              // T_q = A T_{q-1} / q; S += T_q; operand = T_q, or S after the last term
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                const float x = __uint_as_float(dv[e]) * inv;
                const float y = __uint_as_float(sv[e]) + x;
                sv[e] = __float_as_uint(y);
                if (in_b) put_term(i, c0 + e, q < sh.order ? x : y, q < sh.order);
              }
              tmem_st16(tmem + lanes + sreg + (uint32_t)(t * sh.dcol + c0), sv);
            } else if (i < sh.M) {
              // Phi' = S + (E - I) S
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                const int c = c0 + e, b = c < sh.Np ? c : c - sh.Np;
                if (b < sh.N) {
                  const float y = __uint_as_float(sv[e]) + __uint_as_float(dv[e]);
                  const int64_t gi = (c < sh.Np ? 0 : plane) + ((int64_t)w * sh.N + b) * sh.M + i;
                  phi_out[gi] = (double)y;
                  if (phi_out32) phi_out32[gi] = y;
                }
              }
            }
          }
        }
        if (!last) {
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          mbar_arrive(bready);
        }
      }
    }
  }
  __syncthreads();
  // no MMA may still write tensor memory, and no TMA load may still write shared memory
  if (warp == 1 && lane == 0) mbar_wait(done, 0, err, wait_ns);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(sh.tcols)
                 : "memory");
}

// E - I (formed in FP64, rounded to FP32) as split BF16 rows [M][Mp]; padding columns zero
__global__ void k_pack_emI_rows(const double* __restrict__ expK, int M, int Mp,
                                __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const int64_t total = (int64_t)M * Mp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / Mp), j = (int)(e % Mp);
    const float x = j < M ? (float)(expK[(int64_t)i * M + j] - (i == j ? 1.0 : 0.0)) : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[e] = h;
    lo[e] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// rank-2 (j, i) or rank-3 (j, i, z) map over bf16 rows of Mp elements, M x M valid per matrix,
// boxes of 64 x 128 (x 1); the padding j >= M and rows i >= M read as zero (out of bounds)
cudaError_t make_map(CUtensorMap* map, void* base, int M, int Mp, int64_t nz) {
  auto fn = encode_tiled();
  if (!fn) return cudaErrorNotSupported;
  const int rank = nz > 0 ? 3 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)M, (cuuint64_t)M, (cuuint64_t)(nz > 0 ? nz : 1)};
  cuuint64_t strides[2] = {(cuuint64_t)Mp * 2, (cuuint64_t)M * Mp * 2};
  cuuint32_t box[3] = {64u, 128u, 1u};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

TclShape shape_of(const Ctx& c, int nst, int resident) {
  TclShape s{};
  s.ahi = c.tcl_ahi;
  s.alo = c.tcl_alo;
  s.Mp = propagate_tcl_mp(c.M);
  s.M = c.M;
  s.N = c.N;
  s.Np = (c.N + 7) / 8 * 8;
  s.n2 = 2 * s.Np;
  s.MT = (c.M + 127) / 128;
  s.KB = (c.M + 63) / 64;
  s.nst = nst;
  s.bkb = 3 * s.Np * 128;
  s.dcol = (s.n2 + 63) / 64 * 64;
  uint32_t need = (uint32_t)(2 * s.MT * s.dcol), cols = 32;
  while (cols < need) cols <<= 1;
  s.tcols = cols;
  s.order = c.opt.taylor_order;
  s.Nw = c.Nw;
  s.resident = resident;
  s.ring_off = 0;
  s.ares_off = nst * kTile;
  s.bhi_off = s.ares_off + (resident ? 4 * s.KB * kTile : 0);
  s.blo_off = s.bhi_off + s.KB * s.bkb;
  s.bar_off = s.blo_off + s.KB * s.bkb;
  s.smem_bytes = s.bar_off + 8 * (2 * kMaxStages + 5) + 16 + 1024;
  return s;
}

// Launch form: A resident with a 2-stage ring for e^{-dt K/2} - I and 8 epilogue warps, one CTA
// per SM (M <= 128); else A streamed, two CTAs per SM of 4 epilogue warps when a ring of at
// least 4 stages fits 113 KB, otherwise one CTA per SM of 8 epilogue warps with the deepest
// ring that fits.
TclShape plan(const Ctx& c) {
  if (c.M <= 128) {
    const TclShape s = shape_of(c, 2, 1);
    if (s.smem_bytes <= 227 * 1024) return s;
  }
  for (int nst = 8; nst >= 4; --nst) {
    const TclShape s = shape_of(c, nst, 0);
    if (s.smem_bytes <= 113 * 1024) return s;
  }
  for (int nst = kMaxStages; nst >= 2; --nst) {
    const TclShape s = shape_of(c, nst, 0);
    if (s.smem_bytes <= 227 * 1024) return s;
  }
  return shape_of(c, 2, 0);
}

bool two_per_sm(const TclShape& s) { return !s.resident && s.smem_bytes <= 113 * 1024; }

}  // namespace

bool propagate_tcl_ok(const Ctx& c) {
  if (c.M < 1 || c.M > 256 || c.N < 1 || c.N > 32 || c.opt.taylor_order < 1) return false;
  const TclShape s = plan(c);
  return s.smem_bytes <= 227 * 1024 && s.tcols <= 256;
}

int propagate_tcl_mp(int M) { return (M + 7) / 8 * 8; }

cudaError_t prepare_propagate_tcl() {
  cudaError_t e = cudaFuncSetAttribute(k_propagate_tcl<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       227 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_propagate_tcl<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  return e;
}

// Tensor maps of the split A planes (ahi/alo: [2][Nw][M][Mp] bf16) and of E - I (ehi/elo:
// [M][Mp] bf16, packed here from expK).
cudaError_t setup_propagate_tcl(Ctx& c, cudaStream_t s) {
  const int Mp = propagate_tcl_mp(c.M);
  k_pack_emI_rows<<<std::max(1, std::min(152 * 4, (c.M * Mp + 255) / 256)), 256, 0, s>>>(
      c.expK, c.M, Mp, c.tcl_ehi, c.tcl_elo);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap* maps = new CUtensorMap[4];
  e = make_map(&maps[0], c.tcl_ahi, c.M, Mp, 2 * (int64_t)c.Nw);
  if (e == cudaSuccess) e = make_map(&maps[1], c.tcl_alo, c.M, Mp, 2 * (int64_t)c.Nw);
  if (e == cudaSuccess) e = make_map(&maps[2], c.tcl_ehi, c.M, Mp, 0);
  if (e == cudaSuccess) e = make_map(&maps[3], c.tcl_elo, c.M, Mp, 0);
  // without its tensor maps the variant is simply unavailable (taylor_variant_ok checks them)
  delete[] c.tcl_maps;
  c.tcl_maps = e == cudaSuccess ? maps : nullptr;
  if (e != cudaSuccess) delete[] maps;
  return cudaSuccess;
}

// Phi' of every walker from c.phi and the split A planes: out (FP64), out32 (FP32, may be
// null).  With out == c.phi the live walkers are propagated in place and the dead ones left
// as they are.
cudaError_t launch_propagate_tcl(const Ctx& c, double* out, float* out32, cudaStream_t s) {
  if (!propagate_tcl_ok(c) || !c.tcl_maps) return cudaErrorInvalidValue;
  const TclShape sh = plan(c);
  const int* al = out == c.phi ? c.alive : nullptr;
  if (two_per_sm(sh)) {
    k_propagate_tcl<4><<<std::min(c.Nw, 2 * 152), 64 + 32 * 4, sh.smem_bytes, s>>>(
        c.tcl_maps[0], c.tcl_maps[1], c.tcl_maps[2], c.tcl_maps[3], sh, c.phi, out, out32, al,
        c.d_tc_err, kWaitNs);
  } else {
    k_propagate_tcl<8><<<std::min(c.Nw, 152), 64 + 32 * 8, sh.smem_bytes, s>>>(
        c.tcl_maps[0], c.tcl_maps[1], c.tcl_maps[2], c.tcl_maps[3], sh, c.phi, out, out32, al,
        c.d_tc_err, kWaitNs);
  }
  return cudaGetLastError();
}

}  // namespace afq
