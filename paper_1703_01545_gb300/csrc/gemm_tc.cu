// Split-BF16 ("BF16x3") tensor-core GEMM for the Cholesky contractions on sm_103a.
//
//   C[n*ldc + m] = alpha * sum_k (Ahi + Alo)[m][k] (Bhi + Blo)[n][k]     (lo*lo dropped)
//
// A float64 operand x is carried as x ~ hi + lo with hi = bf16(x), lo = bf16(x - hi), so
// each product needs three BF16 MMAs (hi*hi, hi*lo, lo*hi) accumulated in FP32 in tensor
// memory; the product error is about 2^-17 relative instead of BF16's 2^-9.
//
// Structure (one 128 x BN output tile per CTA, 4 warps):
//   warp 0 / lane 0  TMA producer: 128B-swizzled boxes of Ahi, Alo, Bhi, Blo per 64-wide
//                    k slice into a STAGES-deep ring, completion on a "full" mbarrier.
//   warp 1 / lane 0  MMA issuer: per k slice 4 x 3 tcgen05.mma (K = 16 each) into one TMEM
//                    accumulator, then tcgen05.commit frees the stage ("empty" mbarrier);
//                    a final commit signals "done".
//   all 4 warps      epilogue: tcgen05.ld of their 32 TMEM lanes (= 32 output rows m),
//                    scaled by alpha, stored so that a warp writes 32 consecutive m.
// Every mbarrier wait is bounded; on expiry the kernel sets *err, drains what it issued,
// frees its TMEM and returns.  Operand rows are K-major with K padded to a multiple of 64
// (zero-filled), so every TMA box starts on a 128-byte boundary.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "internal.h"
#include "tc_device.cuh"

namespace afq {
namespace {

using namespace tc;

constexpr int BM = 128, BK = 64, NTHREADS = 128;
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s: far beyond any legitimate wait here

template <int BN, int STAGES>
struct TcLayout {
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int BAR_OFFSET = STAGES * STAGE_BYTES;
  static constexpr int SMEM_BYTES = BAR_OFFSET + 256 + 1024;  // barriers + TMEM slot + alignment
};

// Split output of 32 accumulator columns of output row m = i M + j: hi = bf16(x), lo =
// bf16(x - hi) at n * ld + i * Mp + j for columns n = n0 .. n0 + 31 below Nd.
__device__ __forceinline__ void store_split(const SplitOut& so, int m, int n0, int Nd, float alpha,
                                            const uint32_t (&v)[32]) {
  const int i = m / so.M, j = m - i * so.M;
  const int64_t off = (int64_t)i * so.Mp + j;
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    const int n = n0 + q;
    if (n < Nd) {
      const float x = alpha * __uint_as_float(v[q]);
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      so.hi[(int64_t)n * so.ld + off] = h;
      so.lo[(int64_t)n * so.ld + off] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
  }
}

// Lower-triangle block layout of the V_HS rows: tile tm is half h of block q = tm / 2 in the
// order (0,0), (1,0), (1,1), (2,0), ...; block (a, b), a >= b, holds the index pairs
// i in 16 a + [0, 16), j in 16 b + [0, 16), and half h the rows i in 16 a + 8 h + [0, 8).
// Row r of a tile is (i, j) = (16 a + 8 h + r / 16, 16 b + r % 16).
__device__ __forceinline__ void tri_tile(int tm, int& a, int& b, int& h) {
  const int q = tm >> 1;
  h = tm & 1;
  a = (int)((sqrtf(8.f * (float)q + 1.f) - 1.f) * 0.5f);
  while ((a + 1) * (a + 2) / 2 <= q) ++a;
  while (a * (a + 1) / 2 > q) --a;
  b = q - a * (a + 1) / 2;
}

// Split output of 32 accumulator columns of the index pair (i, j) (skipped outside the
// M x M matrix); with `stg`, the pair's hi and lo values also go to column q of the staging
// arrays [32][128] at row r, for the transposed write of the mirror block.
__device__ __forceinline__ void store_split_ij(const SplitOut& so, int i, int j, int n0, int Nd,
                                               float alpha, const uint32_t (&v)[32],
                                               __nv_bfloat16* stg, int r) {
  const bool in = i < so.M && j < so.M;
  const int64_t off = (int64_t)i * so.Mp + j;
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    const int n = n0 + q;
    const float x = alpha * __uint_as_float(v[q]);
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    if (in && n < Nd) {
      so.hi[(int64_t)n * so.ld + off] = h;
      so.lo[(int64_t)n * so.ld + off] = l;
    }
    if (stg) {
      stg[q * BM + r] = h;
      stg[32 * BM + q * BM + r] = l;
    }
  }
}

// The staged 8 x 16 (i, j) half block of 32 columns written transposed: V[j][i0 .. i0 + 7]
// for the 16 j of the block, 16 bytes per (column, j, hi / lo); task t of the 128 epilogue
// threads' 1024.
__device__ __forceinline__ void store_mirror(const SplitOut& so, const __nv_bfloat16* stg, int i0,
                                             int j0, int n0, int Nd, int tid) {
  for (int task = tid; task < 32 * 16 * 2; task += 128) {
    const int q = task >> 5, jj = (task >> 1) & 15, hl = task & 1;
    const int n = n0 + q, j = j0 + jj;
    if (n >= Nd || j >= so.M) continue;
    const __nv_bfloat16* src = stg + hl * 32 * BM + q * BM + jj;   // row r = 16 ii + jj
    __nv_bfloat16* dst = (hl ? so.lo : so.hi) + (int64_t)n * so.ld + (int64_t)j * so.Mp + i0;
    if (i0 + 8 <= so.M) {
      __align__(16) __nv_bfloat16 pk[8];
#pragma unroll
      for (int ii = 0; ii < 8; ++ii) pk[ii] = src[16 * ii];
      *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(pk);
    } else {
      for (int ii = 0; ii < 8 && i0 + ii < so.M; ++ii) dst[ii] = src[16 * ii];
    }
  }
}

// AND of `ok` over the 256 epilogue threads (named barrier 3): they leave the tile loop
// together, so none is left waiting at a staging barrier.
__device__ __forceinline__ bool epilogue_all(bool ok) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, 3, 256, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)ok)
      : "memory");
  return r != 0;
}

// The four warps of epilogue group g (named barrier 1 + g, 128 threads).
__device__ __forceinline__ void group_sync(int g) {
  if (g == 0)
    asm volatile("bar.sync 1, 128;" ::: "memory");
  else
    asm volatile("bar.sync 2, 128;" ::: "memory");
}

template <int BN, int STAGES, class TC>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_gemm_bf16x3_tc(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                     const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                     int Md, int Nd, int nkb, float alpha, TC* __restrict__ C, int64_t ldc,
                     SplitOut so, int* err, uint64_t wait_ns, int skip_producer) {
  using Lay = TcLayout<BN, STAGES>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Lay::BAR_OFFSET);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES),
                 done = smem_u32(bars + 2 * STAGES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"((uint32_t)BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer (skip_producer: self-test of the bounded waits, nothing is issued) ----
    int issued = 0;
    for (int kb = 0; kb < (skip_producer ? 0 : nkb); ++kb) {
      const int s = kb % STAGES, use = kb / STAGES;
      if (kb >= STAGES && !mbar_wait(empty0 + 8 * s, (use - 1) & 1, err, wait_ns)) break;
      const uint32_t st = smem_u32(smem + s * Lay::STAGE_BYTES);
      const uint32_t fb = full0 + 8 * s;
      mbar_expect_tx(fb, Lay::STAGE_BYTES);
      tma_load_2d(st, &tmAh, fb, kb * BK, m0);
      tma_load_2d(st + Lay::A_BYTES, &tmAl, fb, kb * BK, m0);
      tma_load_2d(st + 2 * Lay::A_BYTES, &tmBh, fb, kb * BK, n0);
      tma_load_2d(st + 2 * Lay::A_BYTES + Lay::B_BYTES, &tmBl, fb, kb * BK, n0);
      issued = kb + 1;
    }
    // drain: every issued stage must have landed before the CTA may exit
    for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
      mbar_wait(full0 + 8 * (kb % STAGES), (kb / STAGES) & 1, err, wait_ns);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    const uint32_t idesc = idesc_bf16<BN>();
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES, use = kb / STAGES;
      if (!mbar_wait(full0 + 8 * s, use & 1, err, wait_ns)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t st = smem_u32(smem + s * Lay::STAGE_BYTES);
      const uint64_t ah = sw128_desc(st), al = sw128_desc(st + Lay::A_BYTES);
      const uint64_t bh = sw128_desc(st + 2 * Lay::A_BYTES);
      const uint64_t bl = sw128_desc(st + 2 * Lay::A_BYTES + Lay::B_BYTES);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint64_t dk = (uint64_t)((kk * 32) >> 4);  // advance 16 bf16 inside the swizzle atom
        mma_bf16(tmem, ah + dk, bh + dk, idesc, (kb | kk) != 0);
        mma_bf16(tmem, ah + dk, bl + dk, idesc, 1u);
        mma_bf16(tmem, al + dk, bh + dk, idesc, 1u);
      }
      mma_commit(empty0 + 8 * s);
    }
    mma_commit(done);  // also on an early exit: arrives once the issued MMAs are complete
  }
  __syncwarp();

  // ---- epilogue: TMEM lanes 32*warp .. 32*warp+31 hold output rows m ----
  const bool ok = mbar_wait(done, 0, err, 2 * wait_ns);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncwarp();
  const int m = m0 + warp * 32 + lane;
  if (__all_sync(0xffffffffu, ok && *(volatile int*)err == 0)) {
    for (int c0 = 0; c0 < BN; c0 += 32) {
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (m < Md) {
        if (so.hi) {
          store_split(so, m, n0 + c0, Nd, alpha, v);
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int n = n0 + c0 + j;
            if (n < Nd) C[(int64_t)n * ldc + m] = (TC)(alpha * __uint_as_float(v[j]));
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN)
                 : "memory");
}

// Persistent variant for large outputs (the V_HS contraction): 128 x 256 tiles, grid = one CTA
// per SM looping over tiles, 10 warps.
//   warp 8 / lane 0  TMA producer over all of the CTA's tiles (2-stage ring of 96 KB stages)
//   warp 9 / lane 0  MMA issuer: tile i accumulates into TMEM buffer i & 1 (2 x 256 columns),
//                    commits "tile full" for the epilogue and waits for "tile empty" before it
//                    reuses a buffer
//   warps 0..7       epilogue, two groups of four: group g drains columns 128 g .. 128 g + 127
//                    of buffer i & 1 (warp w reads TMEM lanes 32 (w % 4) ..) while the MMAs of
//                    tile i + 1 run, then arrives on "tile empty"
// Tiles run m-fastest, so consecutive CTAs share B tiles.  Every wait is bounded as above.
constexpr int PBN = 256, PSTAGES = 2, PTHREADS = 320, PEPI = 256;   // PEPI: epilogue threads
struct PLayoutG {
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = PBN * BK * 2;
  static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int STG_OFFSET = PSTAGES * STAGE_BYTES;   // mirror staging per epilogue
  static constexpr int STG_GROUP = 2 * 32 * BM;               // group: hi, lo [32][128] bf16
  static constexpr int BAR_OFFSET = STG_OFFSET + 2 * STG_GROUP * 2;
  static constexpr int SMEM_BYTES = BAR_OFFSET + 256 + 1024;
};

__global__ void __launch_bounds__(PTHREADS, 1)
    k_gemm_bf16x3_tc_persist(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                             const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                             int Md, int Nd, int nkb, float alpha, float* __restrict__ C, int64_t ldc,
                             SplitOut so, int* err, uint64_t wait_ns) {
  using Lay = PLayoutG;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Lay::BAR_OFFSET);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * PSTAGES + 5);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + PSTAGES);
  const uint32_t tfull0 = smem_u32(bars + 2 * PSTAGES), tempty0 = smem_u32(bars + 2 * PSTAGES + 2);
  const uint32_t done = smem_u32(bars + 2 * PSTAGES + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = (Md + BM - 1) / BM, ntiles = mt * ((Nd + PBN - 1) / PBN);

  if (threadIdx.x == 0) {
    for (int s = 0; s < PSTAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, PEPI);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 8) {
    if (lane == 0) {
      // ---- TMA producer ----
      int g = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int m0 = (t % mt) * BM, n0 = (t / mt) * PBN;
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = g % PSTAGES, use = g / PSTAGES;
          if (g >= PSTAGES && !mbar_wait(empty0 + 8 * s, (use - 1) & 1, err, wait_ns)) { ok = false; break; }
          const uint32_t st = smem_u32(smem + s * Lay::STAGE_BYTES);
          const uint32_t fb = full0 + 8 * s;
          mbar_expect_tx(fb, Lay::STAGE_BYTES);
          tma_load_2d(st, &tmAh, fb, kb * BK, m0);
          tma_load_2d(st + Lay::A_BYTES, &tmAl, fb, kb * BK, m0);
          const uint32_t bh = st + 2 * Lay::A_BYTES, bl = bh + Lay::B_BYTES;
          tma_load_2d(bh, &tmBh, fb, kb * BK, n0);
          tma_load_2d(bh + Lay::B_BYTES / 2, &tmBh, fb, kb * BK, n0 + PBN / 2);
          tma_load_2d(bl, &tmBl, fb, kb * BK, n0);
          tma_load_2d(bl + Lay::B_BYTES / 2, &tmBl, fb, kb * BK, n0 + PBN / 2);
        }
      }
      // every issued stage must have landed before the CTA may exit
      for (int q = (g > PSTAGES ? g - PSTAGES : 0); q < g; ++q)
        mbar_wait(full0 + 8 * (q % PSTAGES), (q / PSTAGES) & 1, err, wait_ns);
    }
  } else if (warp == 9) {
    if (lane == 0) {
      // ---- MMA issuer ----
      const uint32_t idesc = idesc_bf16<PBN>();
      int g = 0, i = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++i) {
        const int b = i & 1;
        if (i >= 2 && !mbar_wait(tempty0 + 8 * b, ((i >> 1) - 1) & 1, err, wait_ns)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(b * PBN);
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = g % PSTAGES, use = g / PSTAGES;
          if (!mbar_wait(full0 + 8 * s, use & 1, err, wait_ns)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t st = smem_u32(smem + s * Lay::STAGE_BYTES);
          const uint64_t ah = sw128_desc(st), al = sw128_desc(st + Lay::A_BYTES);
          const uint64_t bh = sw128_desc(st + 2 * Lay::A_BYTES);
          const uint64_t bl = sw128_desc(st + 2 * Lay::A_BYTES + Lay::B_BYTES);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t dk = (uint64_t)((kk * 32) >> 4);
            mma_bf16(d, ah + dk, bh + dk, idesc, (kb | kk) != 0);
            mma_bf16(d, ah + dk, bl + dk, idesc, 1u);
            mma_bf16(d, al + dk, bh + dk, idesc, 1u);
          }
          mma_commit(empty0 + 8 * s);
        }
        if (ok) mma_commit(tfull0 + 8 * b);
      }
      mma_commit(done);   // arrives once every issued MMA has completed
    }
  } else {
    // ---- epilogue: warp w drains TMEM lanes 32 (w % 4) .. + 31 (output rows m) of its
    // group's columns 128 g .. 128 g + 127 ----
    int i = 0;
    const int grp = warp >> 2, wq = warp & 3, cbeg = grp * (PBN / 2), cend = cbeg + PBN / 2;
    __nv_bfloat16* stg =
        reinterpret_cast<__nv_bfloat16*>(smem + Lay::STG_OFFSET) + grp * Lay::STG_GROUP;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int b = i & 1, m0 = (t % mt) * BM, n0 = (t / mt) * PBN;
      const bool ok = mbar_wait(tfull0 + 8 * b, (i >> 1) & 1, err, wait_ns);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (so.tri) {
        if (!epilogue_all(ok)) break;
        // lower-triangle block rows: V[i][j] directly and, off the diagonal, V[j][i] through
        // the staging arrays
        int ta, tb, th;
        tri_tile(t % mt, ta, tb, th);
        const int r = wq * 32 + lane;
        const int ri = 16 * ta + 8 * th + (r >> 4), rj = 16 * tb + (r & 15);
        const bool mirror = ta != tb;
        for (int c0 = cbeg; c0 < cend; c0 += 32) {
          uint32_t v[32];
          tmem_ld32(tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)(b * PBN + c0), v);
          store_split_ij(so, ri, rj, n0 + c0, Nd, alpha, v, mirror ? stg : nullptr, r);
          if (mirror) {
            group_sync(grp);   // the half block's 32 columns are staged
            store_mirror(so, stg, 16 * ta + 8 * th, 16 * tb, n0 + c0, Nd, r);
            group_sync(grp);   // and written: the group's staging arrays are free again
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(tempty0 + 8 * b);
        continue;
      }
      if (!__all_sync(0xffffffffu, ok)) break;
      const int m = m0 + wq * 32 + lane;
      for (int c0 = cbeg; c0 < cend; c0 += 32) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)(b * PBN + c0), v);
        if (m < Md) {
          if (so.hi) {
            store_split(so, m, n0 + c0, Nd, alpha, v);
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int n = n0 + c0 + j;
              if (n < Nd) C[(int64_t)n * ldc + m] = alpha * __uint_as_float(v[j]);
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(tempty0 + 8 * b);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(done, 0, err, wait_ns);   // no MMA may still write TMEM
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u)
                 : "memory");
}

// ---- operand preparation ----

// split rows of a float64 matrix into bf16 hi/lo, K padded with zeros:
// out_{hi,lo}[r][k] for k < Kp; in[r*ld_in + k] for k < K.
__global__ void k_split_bf16(const double* __restrict__ in, int64_t ld_in, int rows, int K, int Kp,
                             __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const int64_t total = (int64_t)rows * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / Kp;
    const int k = (int)(e % Kp);
    const double x = k < K ? in[r * ld_in + k] : 0.0;
    const __nv_bfloat16 h = __float2bfloat16_rn((float)x);
    hi[e] = h;
    lo[e] = __float2bfloat16_rn((float)(x - (double)__bfloat162float(h)));
  }
}

// The lower-triangle block rows (tri_tile) of the V_HS operand: row r of tile r / 128 is the
// index pair (i, j) of row i M + j of `in` ([M^2][ld_in]), zero outside the M x M matrix.
__global__ void k_split_bf16_tri(const double* __restrict__ in, int64_t ld_in, int M, int rows,
                                 int K, int Kp, __nv_bfloat16* __restrict__ hi,
                                 __nv_bfloat16* __restrict__ lo) {
  const int64_t total = (int64_t)rows * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / Kp), k = (int)(e % Kp);
    int a, b, h;
    tri_tile(r >> 7, a, b, h);
    const int i = 16 * a + 8 * h + ((r & 127) >> 4), j = 16 * b + (r & 15);
    const double x = (k < K && i < M && j < M) ? in[((int64_t)i * M + j) * ld_in + k] : 0.0;
    const __nv_bfloat16 hh = __float2bfloat16_rn((float)x);
    hi[e] = hh;
    lo[e] = __float2bfloat16_rn((float)(x - (double)__bfloat162float(hh)));
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

template <int BN, int STAGES, class TC>
cudaError_t launch_tc(const TcOperand& A, const TcOperand& B, int Md, int Nd, float alpha, TC* C,
                      int64_t ldc, int* err, cudaStream_t s, uint64_t wait_ns = kWaitLimitNs,
                      int skip_producer = 0, SplitOut so = SplitOut()) {
  using Lay = TcLayout<BN, STAGES>;
  dim3 grid((Md + BM - 1) / BM, (Nd + BN - 1) / BN);
  if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
  k_gemm_bf16x3_tc<BN, STAGES, TC><<<grid, NTHREADS, Lay::SMEM_BYTES, s>>>(
      A.map_hi, A.map_lo, B.map_hi, B.map_lo, Md, Nd, A.Kp / BK, alpha, C, ldc, so, err, wait_ns,
      skip_producer);
  return cudaGetLastError();
}

}  // namespace

cudaError_t tc_make_operand(TcOperand& op, __nv_bfloat16* hi, __nv_bfloat16* lo, int rows, int Kp,
                            int box_rows) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  // rows must be whole boxes (buffers are padded), so no box ever reaches outside the tensor
  if (Kp % BK != 0 || rows < 1 || rows % box_rows != 0) return cudaErrorInvalidValue;
  op.hi = hi;
  op.lo = lo;
  op.rows = rows;
  op.Kp = Kp;
  cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  for (int q = 0; q < 2; ++q) {
    CUresult r = fn(q == 0 ? &op.map_hi : &op.map_lo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                    q == 0 ? (void*)hi : (void*)lo, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

cudaError_t split_bf16(const double* in, int64_t ld_in, int rows, int K, int Kp, __nv_bfloat16* hi,
                       __nv_bfloat16* lo, cudaStream_t s) {
  const int64_t total = (int64_t)rows * Kp;
  int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 64);
  if (grid < 1) grid = 1;
  k_split_bf16<<<grid, 256, 0, s>>>(in, ld_in, rows, K, Kp, hi, lo);
  return cudaGetLastError();
}

int vhs_tri_rows(int M) {
  const int nb = (M + 15) / 16;
  return nb * (nb + 1) / 2 * 2 * BM;
}

cudaError_t split_bf16_tri(const double* in, int64_t ld_in, int M, int K, int Kp, __nv_bfloat16* hi,
                           __nv_bfloat16* lo, cudaStream_t s) {
  const int rows = vhs_tri_rows(M);
  const int64_t total = (int64_t)rows * Kp;
  int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 64);
  if (grid < 1) grid = 1;
  k_split_bf16_tri<<<grid, 256, 0, s>>>(in, ld_in, M, rows, K, Kp, hi, lo);
  return cudaGetLastError();
}

// The persistent kernel (the only one with the lower-triangle output) takes a product of at
// least two 128 x 256 tiles per SM whose B rows are whole 256-row tiles.
bool tc_persistent_ok(int Md, int Nd, int b_rows) {
  const int64_t tiles = (int64_t)((Md + BM - 1) / BM) * ((Nd + PBN - 1) / PBN);
  return tiles >= 2 * 152 && b_rows % PBN == 0;
}

// A operand boxes are BM = 128 rows; B operand boxes are tc_bn() rows.  Operand buffers
// hold pad_rows(rows) rows (zero-filled beyond `rows`).
int tc_bn() { return 128; }
int tc_pad_rows(int rows) { return (rows + 127) / 128 * 128; }

namespace {
cudaError_t gemm_f32_or_split(const TcOperand& A, const TcOperand& B, int Md, int Nd, float alpha,
                              float* C, int64_t ldc, const SplitOut& so, int* err, cudaStream_t s) {
  if (A.Kp != B.Kp || Md > A.rows || Nd > B.rows) return cudaErrorInvalidValue;
  if (Md <= 0 || Nd <= 0) return cudaSuccess;
  // at least two 128 x 256 tiles per SM: the persistent kernel, whose epilogue overlaps the
  // next tile's MMAs; B tiles of 256 rows stay inside the operand's padded rows (a multiple of
  // 256 here), or read the TMA fill value beyond them
  const int64_t tiles = (int64_t)((Md + BM - 1) / BM) * ((Nd + PBN - 1) / PBN);
  if (so.tri && !tc_persistent_ok(Md, Nd, B.rows)) return cudaErrorInvalidValue;
  if (tc_persistent_ok(Md, Nd, B.rows)) {
    const int grid = (int)std::min<int64_t>(tiles, 152);
    k_gemm_bf16x3_tc_persist<<<grid, PTHREADS, PLayoutG::SMEM_BYTES, s>>>(
        A.map_hi, A.map_lo, B.map_hi, B.map_lo, Md, Nd, A.Kp / BK, alpha, C, ldc, so, err,
        kWaitLimitNs);
    return cudaGetLastError();
  }
  return launch_tc<128, 3, float>(A, B, Md, Nd, alpha, C, ldc, err, s, kWaitLimitNs, 0, so);
}
}  // namespace

cudaError_t gemm_bf16x3(const TcOperand& A, const TcOperand& B, int Md, int Nd, float alpha,
                        float* C, int64_t ldc, int* err, cudaStream_t s) {
  return gemm_f32_or_split(A, B, Md, Nd, alpha, C, ldc, SplitOut(), err, s);
}

cudaError_t gemm_bf16x3_split_out(const TcOperand& A, const TcOperand& B, int Md, int Nd,
                                  float alpha, const SplitOut& so, int* err, cudaStream_t s) {
  if (!so.hi || !so.lo || so.M < 1 || so.Mp < so.M || so.ld < (int64_t)so.M * so.Mp ||
      (so.tri ? vhs_tri_rows(so.M) != Md || so.Mp % 8 != 0 || so.ld % 8 != 0
              : (int64_t)so.M * so.M != Md))
    return cudaErrorInvalidValue;
  return gemm_f32_or_split(A, B, Md, Nd, alpha, nullptr, 0, so, err, s);
}

cudaError_t gemm_bf16x3(const TcOperand& A, const TcOperand& B, int Md, int Nd, float alpha,
                        double* C, int64_t ldc, int* err, cudaStream_t s) {
  if (A.Kp != B.Kp || Md > A.rows || Nd > B.rows) return cudaErrorInvalidValue;
  if (Md <= 0 || Nd <= 0) return cudaSuccess;
  return launch_tc<128, 3, double>(A, B, Md, Nd, alpha, C, ldc, err, s);
}

// Self-test of the bounded waits: the producer issues nothing, so the MMA issuer's wait on
// the first stage expires after `wait_ns`; the kernel must set *err and exit cleanly.
cudaError_t gemm_bf16x3_wait_selftest(const TcOperand& A, const TcOperand& B, int Md, int Nd,
                                      float* C, int64_t ldc, int* err, uint64_t wait_ns,
                                      cudaStream_t s) {
  if (A.Kp != B.Kp || Md > A.rows || Nd > B.rows || Md <= 0 || Nd <= 0) return cudaErrorInvalidValue;
  return launch_tc<128, 3, float>(A, B, Md, Nd, 1.0f, C, ldc, err, s, wait_ns, 1);
}

// Once per process, before any launch or capture: the ring needs ~194 KB of shared memory.
cudaError_t prepare_tc_kernels() {
  static cudaError_t st = cudaErrorNotReady;
  static std::once_flag once;
  std::call_once(once, []() {
    using Lay = TcLayout<128, 3>;
    st = cudaFuncSetAttribute(k_gemm_bf16x3_tc<128, 3, float>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::SMEM_BYTES);
    if (st == cudaSuccess)
      st = cudaFuncSetAttribute(k_gemm_bf16x3_tc<128, 3, double>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::SMEM_BYTES);
    if (st == cudaSuccess)
      st = cudaFuncSetAttribute(k_gemm_bf16x3_tc_persist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                PLayoutG::SMEM_BYTES);
  });
  return st;
}

}  // namespace afq
