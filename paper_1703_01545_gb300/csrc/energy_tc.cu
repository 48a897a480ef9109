// Two-body local energy of the split-precision step on the tensor cores (Eq. 7 with Wick's
// theorem, real and imaginary parts).  For every Cholesky vector g and walker w the matrices
//   T^s_g = Psi_s^T L_g Theta_s          (N_s x N_s per spin, K = M)
// are one GEMM over all (g, w): rows (g, n) of Ltil = Psi^T L_g, columns (w, re/im, n') of
// Theta, both carried as split BF16 (hi + lo, three MMAs per product, FP32 accumulation in
// tensor memory).  The GEMM output never leaves the SM: the epilogue reads each 128 x 256
// accumulator tile from TMEM, stages one walker's rows per warp in shared memory and reduces
//   E2(g, w) = 1/2 [ (sum_s tr T^s_g)^2 - sum_s sum_ab T^s_g[a][b] T^s_g[b][a] ]
// to one partial sum per (row tile, walker); k_energy_tc_reduce adds the row tiles in a
// fixed order and the one-body term sum htil . Theta in FP64.
//
// Orbital padding: each spin block is padded to P2 = max(4, next power of two >= N_s)
// rows, NP = 2 P2 in {8, 16, 32}, so a 128-row tile holds 128 / NP whole Cholesky vectors and
// a warp's 32 TMEM lanes hold whole (g) blocks.  Padded rows and columns are zero, so they
// add nothing; rows past X NP and walkers past Nw are zero-filled operand rows.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "tc_device.cuh"

namespace afq {
namespace {

using namespace tc;

constexpr int EBM = 128, EBN = 256, EBK = 64;
constexpr uint64_t kEWaitNs = 2000000000ull;

__host__ __device__ constexpr int cols_per_group(int NP) { return 2 * NP > 32 ? 2 * NP : 32; }

// One operand stage (A and B of one 64-wide k slice: the next tile's load and MMAs hide behind
// the current tile's epilogue), the epilogue's staging rows (per warp 32 rows x (CW + 1)) and
// the per-tile partial sums of the two tiles in flight: 131-163 KB, one CTA per SM, whose two
// TMEM accumulators take all 512 columns.  8 epilogue warps: two per TMEM lane quadrant, each
// taking half of the tile's column groups.
constexpr int ESTAGES = 1, EWARPS = 8, EPTHREADS = 32 * (EWARPS + 2);
template <int NP>
struct ELayout {
  static constexpr int A_BYTES = EBM * EBK * 2;                 // one of hi / lo
  static constexpr int B_BYTES = EBN * EBK * 2;
  static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int CW = cols_per_group(NP);                 // TMEM columns staged per step
  static constexpr int STG_OFFSET = ESTAGES * STAGE_BYTES;
  static constexpr int STG_BYTES = EWARPS * 32 * (CW + 1) * 4;
  static constexpr int WPT = EBN / (2 * NP);                    // walkers per tile
  static constexpr int RED_OFFSET = STG_OFFSET + STG_BYTES;
  static constexpr int RED_BYTES = 2 * 4 * WPT * 2 * 4;
  static constexpr int BAR_OFFSET = (RED_OFFSET + RED_BYTES + 7) & ~7;
  static constexpr int SMEM_BYTES = BAR_OFFSET + 128 + 1024;    // 9 barriers, flag, TMEM slot, alignment
  static_assert(SMEM_BYTES <= 232448, "one CTA must fit an SM's shared memory");
};

// Operand row r = (unit, n') of a spin-padded block: orbital index or -1 for a padding row.
__device__ __forceinline__ int padded_orbital(int np_, int nu, int nd, int P2) {
  if (np_ < P2) return np_ < nu ? np_ : -1;
  return np_ - P2 < nd ? nu + (np_ - P2) : -1;
}

// A operand: rows (g, n') of Psi_s^T L_g (FP64 Ltil [X][N][M]) split into bf16 hi / lo, K = Kp.
__global__ void k_energy_A(const double* __restrict__ Ltil, int X, int N, int M, int nu, int NP,
                           int Kp, __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const int P2 = NP / 2, nd = N - nu;
  const int64_t total = (int64_t)X * NP * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / Kp;
    const int k = (int)(e % Kp), g = (int)(r / NP), n = padded_orbital((int)(r % NP), nu, nd, P2);
    const double x = (n >= 0 && k < M) ? Ltil[((int64_t)g * N + n) * M + k] : 0.0;
    const __nv_bfloat16 h = __float2bfloat16_rn((float)x);
    hi[e] = h;
    lo[e] = __float2bfloat16_rn((float)(x - (double)__bfloat162float(h)));
  }
}

// B operand: rows (w, p, n') of Theta (FP32 planar [2][Nw][N][M]) split into bf16 hi / lo.
__global__ void k_energy_B(const float* __restrict__ th, int Nw, int N, int M, int nu, int NP,
                           int Kp, __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const int P2 = NP / 2, nd = N - nu;
  const int64_t plane = (int64_t)Nw * N * M, total = (int64_t)Nw * 2 * NP * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / Kp;
    const int k = (int)(e % Kp), w = (int)(r / (2 * NP)), p = (int)((r / NP) & 1);
    const int n = padded_orbital((int)(r % NP), nu, nd, P2);
    const float x = (n >= 0 && k < M) ? th[p * plane + ((int64_t)w * N + n) * M + k] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[e] = h;
    lo[e] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

// Spin-blocked layout (M > 64): one GEMM per spin, so no cross-spin block is computed.  A rows
// (s, g, a), a < P2 of spin s (zero beyond N_s), each spin's rows padded to whole row tiles
// (RTs of them); B rows (s, w, re/im, b) padded to whole column tiles (CTs of them).
__global__ void k_energy_A_spin(const double* __restrict__ Ltil, int X, int N, int M, int nu,
                                int P2, int Kp, int RTs, __nv_bfloat16* __restrict__ hi,
                                __nv_bfloat16* __restrict__ lo) {
  const int64_t per = (int64_t)RTs * EBM, total = 2 * per * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / Kp;
    const int k = (int)(e % Kp), sp = (int)(row / per);
    const int64_t r = row % per;
    const int g = (int)(r / P2), a = (int)(r % P2), ns = sp ? N - nu : nu;
    const double x = (g < X && a < ns && k < M) ? Ltil[((int64_t)g * N + (sp ? nu : 0) + a) * M + k] : 0.0;
    const __nv_bfloat16 h = __float2bfloat16_rn((float)x);
    hi[e] = h;
    lo[e] = __float2bfloat16_rn((float)(x - (double)__bfloat162float(h)));
  }
}

__global__ void k_energy_B_spin(const float* __restrict__ th, int Nw, int N, int M, int nu, int P2,
                                int Kp, int CTs, int nw, __nv_bfloat16* __restrict__ hi,
                                __nv_bfloat16* __restrict__ lo) {
  const int64_t plane = (int64_t)Nw * N * M, per = (int64_t)CTs * EBN;
  const int64_t total = 2 * per * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / Kp;
    const int k = (int)(e % Kp), sp = (int)(row / per);
    const int64_t r = row % per;
    const int w = (int)(r / (2 * P2)), p = (int)((r / P2) & 1), b = (int)(r % P2);
    const int ns = sp ? N - nu : nu;
    const float x = (w < nw && b < ns && k < M)
                        ? th[p * plane + ((int64_t)w * N + (sp ? nu : 0) + b) * M + k] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[e] = h;
    lo[e] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

// Persistent CTAs (one per SM) over the (row tile, column tile) pairs, m-fastest, 10 warps:
//   warp 8 / lane 0  TMA producer
//   warp 9 / lane 0  MMA issuer: per 64-wide k slice 4 x 3 tcgen05.mma (K = 16, N = 256) into
//                    TMEM buffer i & 1 of the CTA's i-th tile, then "tile full"
//   warps 0..7       epilogue: warp w reads TMEM lanes 32 (w % 4) .. (rows (g, a)) of buffer
//                    i & 1, column groups of half w / 4, while the next tile's load and MMAs
//                    run; "tile empty" once the rows are read; the 8 warps meet at a named
//                    barrier to add their partial sums
// part[(tile_row * 2 + re/im) * NwP + w] = sum over the tile's g of E2(g, w).
// Every mbarrier wait is bounded; on expiry *err is set, the epilogue warps stop together
// (a shared flag read after their barrier), the CTA drains what it issued and frees its TMEM.
// SPIN: spin-blocked layout (rows of one spin block per g, NP = P2): tiles t = (s, column
// tile, row tile), the exchange over the whole block, and the traces tr T^s_g to trs (the
// reduction forms the Coulomb term from both spins); otherwise both spins per g (NP = 2 P2),
// exchange per spin block and the Coulomb term.
template <int NP, bool SPIN>
__global__ void __launch_bounds__(EPTHREADS, 1)
    k_energy_tc(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                int nkb, int RT, int CT, float* __restrict__ part, int NwP, int* err,
                uint64_t wait_ns, float2* __restrict__ trs, int X, int Nw) {
  using Lay = ELayout<NP>;
  constexpr int CW = Lay::CW, WPT = Lay::WPT, P2 = SPIN ? NP : NP / 2, WPG = CW / (2 * NP);
  extern __shared__ uint8_t esm_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(esm_raw) + 1023) &
                                             ~uintptr_t(1023));
  float* stg = reinterpret_cast<float*>(smem + Lay::STG_OFFSET);
  float* red = reinterpret_cast<float*>(smem + Lay::RED_OFFSET);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Lay::BAR_OFFSET);
  volatile int* s_fail = reinterpret_cast<volatile int*>(bars + 9);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 10);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + 2);
  const uint32_t tfull0 = smem_u32(bars + 4), tempty0 = smem_u32(bars + 6), done = smem_u32(bars + 8);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = (SPIN ? 2 : 1) * RT * CT;
  // tile t: spin block sp, row tile rt, column tile ct (rows and columns of the same spin)
  auto tile_of = [&](int t, int& m0, int& n0, int& rt_all, int& ct) {
    const int sp = t / (RT * CT), r = t % (RT * CT), rt = r % RT;
    ct = r / RT;
    rt_all = sp * RT + rt;
    m0 = rt_all * EBM;
    n0 = (sp * CT + ct) * EBN;
  };

  if (threadIdx.x == 0) {
    for (int q = 0; q < 2; ++q) {
      mbar_init(full0 + 8 * q, 1);
      mbar_init(empty0 + 8 * q, 1);
      mbar_init(tfull0 + 8 * q, 1);
      mbar_init(tempty0 + 8 * q, 32 * EWARPS);
    }
    mbar_init(done, 1);
    *s_fail = 0;
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

  if (warp == EWARPS) {
    if (lane == 0) {
      // ---- TMA producer ----
      int g = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int m0, n0, rt_all, ct;
        tile_of(t, m0, n0, rt_all, ct);
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = g % ESTAGES, use = g / ESTAGES;
          if (g >= ESTAGES && !mbar_wait(empty0 + 8 * s, (use - 1) & 1, err, wait_ns)) { ok = false; break; }
          const uint32_t st = smem_u32(smem + s * Lay::STAGE_BYTES), fb = full0 + 8 * s;
          const int kx = kb * EBK;
          mbar_expect_tx(fb, Lay::STAGE_BYTES);
          tma_load_2d(st, &tmAh, fb, kx, m0);
          tma_load_2d(st + Lay::A_BYTES, &tmAl, fb, kx, m0);
          const uint32_t bh = st + 2 * Lay::A_BYTES, bl = bh + Lay::B_BYTES;
          tma_load_2d(bh, &tmBh, fb, kx, n0);
          tma_load_2d(bh + Lay::B_BYTES / 2, &tmBh, fb, kx, n0 + EBN / 2);
          tma_load_2d(bl, &tmBl, fb, kx, n0);
          tma_load_2d(bl + Lay::B_BYTES / 2, &tmBl, fb, kx, n0 + EBN / 2);
        }
      }
      // every issued stage must have landed before the CTA may exit
      for (int q = (g > ESTAGES ? g - ESTAGES : 0); q < g; ++q)
        mbar_wait(full0 + 8 * (q % ESTAGES), (q / ESTAGES) & 1, err, wait_ns);
    }
  } else if (warp == EWARPS + 1) {
    if (lane == 0) {
      // ---- MMA issuer ----
      const uint32_t idesc = idesc_bf16<EBN>();
      int g = 0, i = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++i) {
        const int b = i & 1;
        if (i >= 2 && !mbar_wait(tempty0 + 8 * b, ((i >> 1) - 1) & 1, err, wait_ns)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(b * EBN);
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = g % ESTAGES, use = g / ESTAGES;
          if (!mbar_wait(full0 + 8 * s, use & 1, err, wait_ns)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t st = smem_u32(smem + s * Lay::STAGE_BYTES);
          const uint64_t ah = sw128_desc(st), al = sw128_desc(st + Lay::A_BYTES);
          const uint64_t bh = sw128_desc(st + 2 * Lay::A_BYTES);
          const uint64_t bl = sw128_desc(st + 2 * Lay::A_BYTES + Lay::B_BYTES);
#pragma unroll
          for (int kk = 0; kk < EBK / 16; ++kk) {
            const uint64_t dk = (uint64_t)((kk * 32) >> 4);   // 16 bf16 = 32 bytes inside the atom
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
    // ---- epilogue ----
    constexpr int NG = EBN / CW, NGH = NG / 2;   // column groups per tile, per half
    float* S = stg + warp * 32 * (CW + 1);
    const int quad = warp & 3, half = warp >> 2;
    const int a = lane % NP, gl = lane / NP, s0 = (SPIN || a < P2) ? 0 : P2;
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      int m0_, n0_, rt_all, ct_t;
      tile_of(t, m0_, n0_, rt_all, ct_t);
      const int b = i & 1;
      float* rb = red + b * (4 * WPT * 2);
      const bool ok = mbar_wait(tfull0 + 8 * b, (i >> 1) & 1, err, wait_ns);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (__all_sync(0xffffffffu, ok)) {
        for (int gg = 0; gg < NGH; ++gg) {
          const int grp = half * NGH + gg;
          float rowv[CW];   // this lane's row (g, a) of the group: its own T[a][.]
#pragma unroll
          for (int h = 0; h < CW / 32; ++h) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * EBN + grp * CW + 32 * h), v);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              rowv[32 * h + j] = __uint_as_float(v[j]);
              S[lane * (CW + 1) + 32 * h + j] = rowv[32 * h + j];
            }
          }
          __syncwarp();
#pragma unroll
          for (int wi = 0; wi < WPG; ++wi) {
            const int cb = wi * 2 * NP;
            const float* colp = S + gl * NP * (CW + 1) + cb + a;        // T[.][a]
            float exr = 0.f, exi = 0.f;
#pragma unroll
            for (int j = 0; j < P2; ++j) {
              // T[a][s0 + j] T[s0 + j][a] over the lane's spin block
              const float tr = s0 ? rowv[cb + P2 + j] : rowv[cb + j];
              const float ti = s0 ? rowv[cb + NP + P2 + j] : rowv[cb + NP + j];
              const float ur = colp[(s0 + j) * (CW + 1)], ui = colp[(s0 + j) * (CW + 1) + NP];
              exr = fmaf(tr, ur, fmaf(-ti, ui, exr));
              exi = fmaf(tr, ui, fmaf(ti, ur, exi));
            }
            float dr = S[lane * (CW + 1) + cb + a], di = S[lane * (CW + 1) + cb + NP + a];   // T[a][a]
#pragma unroll
            for (int o = NP / 2; o > 0; o >>= 1) {                     // sums over the g block
              exr += __shfl_xor_sync(0xffffffffu, exr, o);
              exi += __shfl_xor_sync(0xffffffffu, exi, o);
              dr += __shfl_xor_sync(0xffffffffu, dr, o);
              di += __shfl_xor_sync(0xffffffffu, di, o);
            }
            // the Coulomb term (sum_s tr T^s)^2 needs both spins: in the spin-blocked layout
            // the traces tr T^s_g go to trs and the reduction combines the spins
            if (SPIN && a == 0) {
              const int sp = rt_all / RT;
              const int g = ((rt_all - sp * RT) * EBM + quad * 32 + lane) / NP;
              const int w = ct_t * WPT + grp * WPG + wi;
              if (g < X && w < Nw) trs[((int64_t)sp * Nw + w) * X + g] = make_float2(dr, di);
            }
            float er = a == 0 ? 0.5f * ((SPIN ? 0.f : dr * dr - di * di) - exr) : 0.f;
            float ei = a == 0 ? 0.5f * ((SPIN ? 0.f : 2.f * dr * di) - exi) : 0.f;
#pragma unroll
            for (int o = NP; o < 32; o <<= 1) {                        // over the warp's g blocks
              er += __shfl_xor_sync(0xffffffffu, er, o);
              ei += __shfl_xor_sync(0xffffffffu, ei, o);
            }
            if (lane == 0) {
              rb[(quad * WPT + grp * WPG + wi) * 2] = er;
              rb[(quad * WPT + grp * WPG + wi) * 2 + 1] = ei;
            }
          }
          __syncwarp();
        }
      } else if (lane == 0) {
        *s_fail = 1;
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(tempty0 + 8 * b);
      asm volatile("bar.sync 1, %0;" ::"n"(32 * EWARPS) : "memory");   // the epilogue warps
      if (*s_fail) break;
      if (threadIdx.x < WPT) {
        const int w = ct_t * WPT + threadIdx.x, rt = rt_all;
        float sr = 0.f, si = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          sr += rb[(q * WPT + threadIdx.x) * 2];
          si += rb[(q * WPT + threadIdx.x) * 2 + 1];
        }
        part[(int64_t)(2 * rt) * NwP + w] = sr;
        part[(int64_t)(2 * rt + 1) * NwP + w] = si;
      }
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

// Single k slice (M <= 64): the column tile of Theta stays in shared memory while the CTA
// runs a group of RG row tiles of Psi^T L_g through it, so the operand stream is one B tile
// per group plus the small A tiles (the per-tile form re-reads B for every row tile).
// Work item = (column tile, row group); each walker's partial sums over the group's row tiles
// add up in the epilogue and part[(group * 2 + re/im) * NwP + w] receives them.  Warp roles as
// in k_energy_tc (with bres_ewarps(NP) epilogue warps); shared memory: B (64 KB), 2 A stages
// (32 KB each), staging, partials.
// Epilogue warps of the B-resident form: four per TMEM lane quadrant (two for NP = 32, whose
// staging rows are twice as wide).
__host__ __device__ constexpr int bres_ewarps(int NP) { return NP == 32 ? 8 : 16; }

template <int NP>
struct EBLayout {
  static constexpr int EW = bres_ewarps(NP), THREADS = 32 * (EW + 2);
  static constexpr int A_BYTES = EBM * EBK * 2;                 // one of hi / lo
  static constexpr int B_BYTES = EBN * EBK * 2;
  static constexpr int A_OFFSET = 2 * B_BYTES;
  static constexpr int A_STAGE = 2 * A_BYTES;
  static constexpr int CW = cols_per_group(NP);
  static constexpr int STG_OFFSET = A_OFFSET + 2 * A_STAGE;
  static constexpr int STG_BYTES = EW * 32 * (CW + 1) * 4;
  static constexpr int WPT = EBN / (2 * NP);
  static constexpr int RED_OFFSET = STG_OFFSET + STG_BYTES;
  static constexpr int RED_BYTES = 2 * 4 * WPT * 2 * 4;
  static constexpr int BAR_OFFSET = (RED_OFFSET + RED_BYTES + 7) & ~7;
  static constexpr int SMEM_BYTES = BAR_OFFSET + 128 + 1024;    // 11 barriers, flag, TMEM slot, alignment
  static_assert(SMEM_BYTES <= 232448, "one CTA must fit an SM's shared memory");
};

template <int NP>
__global__ void __launch_bounds__(EBLayout<NP>::THREADS, 1)
    k_energy_tc_bres(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                     const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                     int RT, int CT, int RG, int NG, float* __restrict__ part, int NwP, int* err,
                     uint64_t wait_ns) {
  using Lay = EBLayout<NP>;
  constexpr int CW = Lay::CW, WPT = Lay::WPT, P2 = NP / 2, WPG = CW / (2 * NP), EW = Lay::EW;
  extern __shared__ uint8_t esm_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(esm_raw) + 1023) &
                                             ~uintptr_t(1023));
  float* stg = reinterpret_cast<float*>(smem + Lay::STG_OFFSET);
  float* red = reinterpret_cast<float*>(smem + Lay::RED_OFFSET);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Lay::BAR_OFFSET);
  volatile int* s_fail = reinterpret_cast<volatile int*>(bars + 11);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 12);
  const uint32_t bfull = smem_u32(bars), bempty = smem_u32(bars + 1);
  const uint32_t full0 = smem_u32(bars + 2), empty0 = smem_u32(bars + 4);
  const uint32_t tfull0 = smem_u32(bars + 6), tempty0 = smem_u32(bars + 8), done = smem_u32(bars + 10);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nitems = CT * NG;
  const uint32_t sbase = smem_u32(smem);

  if (threadIdx.x == 0) {
    mbar_init(bfull, 1);
    mbar_init(bempty, 1);
    for (int q = 0; q < 2; ++q) {
      mbar_init(full0 + 8 * q, 1);
      mbar_init(empty0 + 8 * q, 1);
      mbar_init(tfull0 + 8 * q, 1);
      mbar_init(tempty0 + 8 * q, 32 * EW);
    }
    mbar_init(done, 1);
    *s_fail = 0;
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

  if (warp == EW) {
    if (lane == 0) {
      // ---- TMA producer: B once per item (after the previous item's MMAs), A per row tile ----
      int ga = 0, j = 0;
      bool ok = true;
      for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x, ++j) {
        const int ct = it / NG, rg = it % NG, n0 = ct * EBN;
        const int r0 = rg * RG, r1 = min(RT, r0 + RG);
        if (j > 0 && !mbar_wait(bempty, (j - 1) & 1, err, wait_ns)) break;
        mbar_expect_tx(bfull, 2 * Lay::B_BYTES);
        tma_load_2d(sbase, &tmBh, bfull, 0, n0);
        tma_load_2d(sbase + Lay::B_BYTES / 2, &tmBh, bfull, 0, n0 + EBN / 2);
        tma_load_2d(sbase + Lay::B_BYTES, &tmBl, bfull, 0, n0);
        tma_load_2d(sbase + Lay::B_BYTES + Lay::B_BYTES / 2, &tmBl, bfull, 0, n0 + EBN / 2);
        for (int rt = r0; rt < r1; ++rt, ++ga) {
          const int s = ga & 1, use = ga >> 1;
          if (ga >= 2 && !mbar_wait(empty0 + 8 * s, (use - 1) & 1, err, wait_ns)) { ok = false; break; }
          const uint32_t st = sbase + Lay::A_OFFSET + s * Lay::A_STAGE, fb = full0 + 8 * s;
          mbar_expect_tx(fb, Lay::A_STAGE);
          tma_load_2d(st, &tmAh, fb, 0, rt * EBM);
          tma_load_2d(st + Lay::A_BYTES, &tmAl, fb, 0, rt * EBM);
        }
      }
      // every issued copy must have landed before the CTA may exit
      if (j > 0) mbar_wait(bfull, (j - 1) & 1, err, wait_ns);
      for (int q = (ga > 2 ? ga - 2 : 0); q < ga; ++q)
        mbar_wait(full0 + 8 * (q & 1), (q >> 1) & 1, err, wait_ns);
    }
  } else if (warp == EW + 1) {
    if (lane == 0) {
      // ---- MMA issuer ----
      const uint32_t idesc = idesc_bf16<EBN>();
      const uint64_t bh = sw128_desc(sbase), bl = sw128_desc(sbase + Lay::B_BYTES);
      int ga = 0, i = 0, j = 0;
      bool ok = true;
      for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x, ++j) {
        const int rg = it % NG, r0 = rg * RG, r1 = min(RT, r0 + RG);
        if (!mbar_wait(bfull, j & 1, err, wait_ns)) break;
        for (int rt = r0; rt < r1; ++rt, ++ga, ++i) {
          const int b = i & 1, s = ga & 1;
          if (i >= 2 && !mbar_wait(tempty0 + 8 * b, ((i >> 1) - 1) & 1, err, wait_ns)) { ok = false; break; }
          if (!mbar_wait(full0 + 8 * s, (ga >> 1) & 1, err, wait_ns)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t st = sbase + Lay::A_OFFSET + s * Lay::A_STAGE;
          const uint64_t ah = sw128_desc(st), al = sw128_desc(st + Lay::A_BYTES);
          const uint32_t d = tmem + (uint32_t)(b * EBN);
#pragma unroll
          for (int kk = 0; kk < EBK / 16; ++kk) {
            const uint64_t dk = (uint64_t)((kk * 32) >> 4);
            mma_bf16(d, ah + dk, bh + dk, idesc, kk != 0);
            mma_bf16(d, ah + dk, bl + dk, idesc, 1u);
            mma_bf16(d, al + dk, bh + dk, idesc, 1u);
          }
          mma_commit(empty0 + 8 * s);
          mma_commit(tfull0 + 8 * b);
        }
        mma_commit(bempty);   // the item's MMAs are done with B once this arrives
      }
      mma_commit(done);
    }
  } else {
    // ---- epilogue ----
    constexpr int NPART = EW / 4, NGR = EBN / CW, NGH = NGR / NPART;   // column groups per warp
    float* S = stg + warp * 32 * (CW + 1);
    const int quad = warp & 3, half = warp >> 2;
    const int a = lane % NP, gl = lane / NP, s0 = a < P2 ? 0 : P2;
    int i = 0;
    bool stop = false;
    for (int it = blockIdx.x; it < nitems && !stop; it += gridDim.x) {
      const int ct = it / NG, rg = it % NG, r0 = rg * RG, r1 = min(RT, r0 + RG);
      float accr = 0.f, acci = 0.f;   // threads < WPT: walker ct * WPT + threadIdx.x
      for (int rt = r0; rt < r1; ++rt, ++i) {
        const int b = i & 1;
        float* rb = red + b * (4 * WPT * 2);
        const bool ok = mbar_wait(tfull0 + 8 * b, (i >> 1) & 1, err, wait_ns);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (__all_sync(0xffffffffu, ok)) {
          for (int gg = 0; gg < NGH; ++gg) {
            const int grp = half * NGH + gg;
            float rowv[CW];
#pragma unroll
            for (int h = 0; h < CW / 32; ++h) {
              uint32_t v[32];
              tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * EBN + grp * CW + 32 * h), v);
#pragma unroll
              for (int q = 0; q < 32; ++q) {
                rowv[32 * h + q] = __uint_as_float(v[q]);
                S[lane * (CW + 1) + 32 * h + q] = rowv[32 * h + q];
              }
            }
            __syncwarp();
#pragma unroll
            for (int wi = 0; wi < WPG; ++wi) {
              const int cb = wi * 2 * NP;
              const float* colp = S + gl * NP * (CW + 1) + cb + a;        // T[.][a]
              float exr = 0.f, exi = 0.f;
#pragma unroll
              for (int q = 0; q < P2; ++q) {
                // T[a][s0 + q] T[s0 + q][a] over the lane's spin block
                const float tr = s0 ? rowv[cb + P2 + q] : rowv[cb + q];
                const float ti = s0 ? rowv[cb + NP + P2 + q] : rowv[cb + NP + q];
                const float ur = colp[(s0 + q) * (CW + 1)], ui = colp[(s0 + q) * (CW + 1) + NP];
                exr = fmaf(tr, ur, fmaf(-ti, ui, exr));
                exi = fmaf(tr, ui, fmaf(ti, ur, exi));
              }
              float dr = S[lane * (CW + 1) + cb + a], di = S[lane * (CW + 1) + cb + NP + a];   // T[a][a]
#pragma unroll
              for (int o = NP / 2; o > 0; o >>= 1) {
                exr += __shfl_xor_sync(0xffffffffu, exr, o);
                exi += __shfl_xor_sync(0xffffffffu, exi, o);
                dr += __shfl_xor_sync(0xffffffffu, dr, o);
                di += __shfl_xor_sync(0xffffffffu, di, o);
              }
              float er = a == 0 ? 0.5f * (dr * dr - di * di - exr) : 0.f;
              float ei = a == 0 ? 0.5f * (2.f * dr * di - exi) : 0.f;
#pragma unroll
              for (int o = NP; o < 32; o <<= 1) {
                er += __shfl_xor_sync(0xffffffffu, er, o);
                ei += __shfl_xor_sync(0xffffffffu, ei, o);
              }
              if (lane == 0) {
                rb[(quad * WPT + grp * WPG + wi) * 2] = er;
                rb[(quad * WPT + grp * WPG + wi) * 2 + 1] = ei;
              }
            }
            __syncwarp();
          }
        } else if (lane == 0) {
          *s_fail = 1;
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(tempty0 + 8 * b);
        asm volatile("bar.sync 1, %0;" ::"n"(32 * EW) : "memory");   // the epilogue warps
        if (*s_fail) { stop = true; break; }
        if (threadIdx.x < WPT)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            accr += rb[(q * WPT + threadIdx.x) * 2];
            acci += rb[(q * WPT + threadIdx.x) * 2 + 1];
          }
      }
      if (!stop && threadIdx.x < WPT) {
        const int w = ct * WPT + threadIdx.x;
        part[(int64_t)(2 * rg) * NwP + w] = accr;
        part[(int64_t)(2 * rg + 1) * NwP + w] = acci;
      }
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

__device__ __forceinline__ void tmem_ld32_nw(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
        "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
        "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld_e() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Spin-blocked form with two k slices (64 < M <= 128): a CTA keeps the whole Theta column tile
// of one spin block resident (both k slices, hi and lo: 128 KB) and streams a group of RG row
// tiles of L-tilde through a 2-stage ring of one k slice each, so the operand traffic is one
// Theta tile per item plus the row tiles (the per-tile form reloads both for every tile).
// Work item = (spin, column tile, row group); each walker's exchange sums over the item's row
// tiles add up in the epilogue, part[(spin * NG + group) * 2 + re/im) * NwP + w]; the traces
// tr T^s_g of each tile go to trs.  Warp roles and epilogue as in k_energy_tc (8 epilogue
// warps, rows staged with one word of padding); 227 KB of shared memory.
template <int NP>
struct ES2Layout {
  static constexpr int NKB = 2;
  static constexpr int A_BYTES = EBM * EBK * 2;                 // one k slice, one of hi / lo
  static constexpr int B_BYTES = EBN * EBK * 2;
  static constexpr int B_REGION = NKB * 2 * B_BYTES;            // (k slice, hi / lo)
  static constexpr int A_OFFSET = B_REGION;
  static constexpr int A_STAGE = 2 * A_BYTES;
  static constexpr int CW = 2 * NP;                             // one walker's re | im columns
  static_assert(CW == 32, "the swizzled staging assumes 32 columns per group");
  static constexpr int STG_OFFSET = A_OFFSET + 2 * A_STAGE;
  static constexpr int STG_BYTES = EWARPS * 32 * 33 * 4;
  static constexpr int WPT = EBN / (2 * NP);
  static constexpr int RED_OFFSET = STG_OFFSET + STG_BYTES;
  static constexpr int RED_BYTES = 2 * 4 * WPT * 2 * 4;
  static constexpr int BAR_OFFSET = (RED_OFFSET + RED_BYTES + 7) & ~7;
  static constexpr int SMEM_BYTES = BAR_OFFSET + 128 + 1024;
  static_assert(SMEM_BYTES <= 232448, "one CTA must fit an SM's shared memory");
};

template <int NP>
__global__ void __launch_bounds__(EPTHREADS, 1)
    k_energy_tc_spin2(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                      const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                      int RT, int CT, int RG, int NG, float* __restrict__ part, int NwP, int* err,
                      uint64_t wait_ns, float2* __restrict__ trs, int X, int Nw) {
  using Lay = ES2Layout<NP>;
  constexpr int WPT = Lay::WPT, NKB = Lay::NKB;
  extern __shared__ uint8_t esm_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(esm_raw) + 1023) &
                                             ~uintptr_t(1023));
  float* stg = reinterpret_cast<float*>(smem + Lay::STG_OFFSET);
  float* red = reinterpret_cast<float*>(smem + Lay::RED_OFFSET);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Lay::BAR_OFFSET);
  volatile int* s_fail = reinterpret_cast<volatile int*>(bars + 11);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 12);
  const uint32_t bfull = smem_u32(bars), bempty = smem_u32(bars + 1);
  const uint32_t full0 = smem_u32(bars + 2), empty0 = smem_u32(bars + 4);
  const uint32_t tfull0 = smem_u32(bars + 6), tempty0 = smem_u32(bars + 8), done = smem_u32(bars + 10);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nitems = 2 * CT * NG;
  const uint32_t sbase = smem_u32(smem);
  // item -> spin, column tile, row tiles [r0, r1)
  auto item_of = [&](int it, int& sp, int& ct, int& rg, int& r0, int& r1) {
    sp = it / (CT * NG);
    const int rem = it - sp * CT * NG;
    ct = rem / NG;
    rg = rem - ct * NG;
    r0 = rg * RG;
    r1 = min(RT, r0 + RG);
  };

  if (threadIdx.x == 0) {
    mbar_init(bfull, 1);
    mbar_init(bempty, 1);
    for (int q = 0; q < 2; ++q) {
      mbar_init(full0 + 8 * q, 1);
      mbar_init(empty0 + 8 * q, 1);
      mbar_init(tfull0 + 8 * q, 1);
      mbar_init(tempty0 + 8 * q, 32 * EWARPS);
    }
    mbar_init(done, 1);
    *s_fail = 0;
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

  if (warp == EWARPS) {
    if (lane == 0) {
      // ---- TMA producer: the Theta tile once per item (after the previous item's MMAs), one
      // k slice of the L-tilde row tile per ring stage ----
      int ga = 0, j = 0;
      bool ok = true;
      for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x, ++j) {
        int sp, ct, rg, r0, r1;
        item_of(it, sp, ct, rg, r0, r1);
        const int n0 = (sp * CT + ct) * EBN;
        if (j > 0 && !mbar_wait(bempty, (j - 1) & 1, err, wait_ns)) break;
        mbar_expect_tx(bfull, Lay::B_REGION);
        for (int kb = 0; kb < NKB; ++kb)
          for (int lo = 0; lo < 2; ++lo) {
            const uint32_t dst = sbase + (uint32_t)((kb * 2 + lo) * Lay::B_BYTES);
            tma_load_2d(dst, lo ? &tmBl : &tmBh, bfull, kb * EBK, n0);
            tma_load_2d(dst + Lay::B_BYTES / 2, lo ? &tmBl : &tmBh, bfull, kb * EBK, n0 + EBN / 2);
          }
        for (int rt = r0; rt < r1 && ok; ++rt)
          for (int kb = 0; kb < NKB; ++kb, ++ga) {
            const int s = ga & 1, use = ga >> 1;
            if (ga >= 2 && !mbar_wait(empty0 + 8 * s, (use - 1) & 1, err, wait_ns)) { ok = false; break; }
            const uint32_t st = sbase + Lay::A_OFFSET + s * Lay::A_STAGE, fb = full0 + 8 * s;
            const int m0 = (sp * RT + rt) * EBM;
            mbar_expect_tx(fb, Lay::A_STAGE);
            tma_load_2d(st, &tmAh, fb, kb * EBK, m0);
            tma_load_2d(st + Lay::A_BYTES, &tmAl, fb, kb * EBK, m0);
          }
      }
      // every issued copy must have landed before the CTA may exit
      if (j > 0) mbar_wait(bfull, (j - 1) & 1, err, wait_ns);
      for (int q = (ga > 2 ? ga - 2 : 0); q < ga; ++q)
        mbar_wait(full0 + 8 * (q & 1), (q >> 1) & 1, err, wait_ns);
    }
  } else if (warp == EWARPS + 1) {
    if (lane == 0) {
      // ---- MMA issuer ----
      const uint32_t idesc = idesc_bf16<EBN>();
      int ga = 0, i = 0, j = 0;
      bool ok = true;
      for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x, ++j) {
        int sp, ct, rg, r0, r1;
        item_of(it, sp, ct, rg, r0, r1);
        if (!mbar_wait(bfull, j & 1, err, wait_ns)) break;
        for (int rt = r0; rt < r1 && ok; ++rt, ++i) {
          const int b = i & 1;
          if (i >= 2 && !mbar_wait(tempty0 + 8 * b, ((i >> 1) - 1) & 1, err, wait_ns)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t d = tmem + (uint32_t)(b * EBN);
          for (int kb = 0; kb < NKB; ++kb, ++ga) {
            const int s = ga & 1;
            if (!mbar_wait(full0 + 8 * s, (ga >> 1) & 1, err, wait_ns)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t st = sbase + Lay::A_OFFSET + s * Lay::A_STAGE;
            const uint64_t ah = sw128_desc(st), al = sw128_desc(st + Lay::A_BYTES);
            const uint64_t bh = sw128_desc(sbase + (uint32_t)(kb * 2 * Lay::B_BYTES));
            const uint64_t bl = sw128_desc(sbase + (uint32_t)((kb * 2 + 1) * Lay::B_BYTES));
#pragma unroll
            for (int kk = 0; kk < EBK / 16; ++kk) {
              const uint64_t dk = (uint64_t)((kk * 32) >> 4);
              mma_bf16(d, ah + dk, bh + dk, idesc, (kb | kk) != 0);
              mma_bf16(d, ah + dk, bl + dk, idesc, 1u);
              mma_bf16(d, al + dk, bh + dk, idesc, 1u);
            }
            mma_commit(empty0 + 8 * s);
          }
          if (ok) mma_commit(tfull0 + 8 * b);
        }
        mma_commit(bempty);   // the item's MMAs are done with the Theta tile once this arrives
      }
      mma_commit(done);
    }
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. (rows (g, a)), column groups of half
    // w / 4; per group one walker's re | im columns ----
    constexpr int NGR = EBN / 32, NGH = NGR / 2;
    float* S = stg + warp * 32 * 33;
    const int quad = warp & 3, half = warp >> 2;
    const int a = lane % NP, gl = lane / NP;
    int i = 0;
    bool stop = false;
    for (int it = blockIdx.x; it < nitems && !stop; it += gridDim.x) {
      int sp, ct, rg, r0, r1;
      item_of(it, sp, ct, rg, r0, r1);
      float accr = 0.f, acci = 0.f;   // threads < WPT: walker ct * WPT + threadIdx.x
      for (int rt = r0; rt < r1; ++rt, ++i) {
        const int b = i & 1;
        float* rb = red + b * (4 * WPT * 2);
        const bool ok = mbar_wait(tfull0 + 8 * b, (i >> 1) & 1, err, wait_ns);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (__all_sync(0xffffffffu, ok)) {
          const int g = (rt * EBM + quad * 32 + lane) / NP;
          const uint32_t tq = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * EBN + half * NGH * 32);
          // group gg + 1's TMEM load is in flight while group gg is reduced
          uint32_t va[32], vb[32];
          tmem_ld32_nw(tq, va);
          tmem_wait_ld_e();
#pragma unroll
          for (int gg = 0; gg < NGH; ++gg) {
            uint32_t(&v)[32] = (gg & 1) ? vb : va;
            if (gg + 1 < NGH) tmem_ld32_nw(tq + (uint32_t)(32 * (gg + 1)), (gg & 1) ? va : vb);
            const int grp = half * NGH + gg;
            // staged rows of 33 words: the row writes and the column reads below fall in
            // distinct banks
#pragma unroll
            for (int q = 0; q < 32; ++q) S[lane * 33 + q] = __uint_as_float(v[q]);
            __syncwarp();
            // exchange of (g, w): sum_b T[a][b] T[b][a], T[b][a] from row (gl NP + b), column a
            const float* colp = S + gl * NP * 33 + a;
            float exr0 = 0.f, exi0 = 0.f, exr1 = 0.f, exi1 = 0.f;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
              const float ur = colp[q * 33], ui = colp[q * 33 + NP];
              const float tr = __uint_as_float(v[q]), ti = __uint_as_float(v[NP + q]);
              if (q & 1) {
                exr1 = fmaf(tr, ur, fmaf(-ti, ui, exr1));
                exi1 = fmaf(tr, ui, fmaf(ti, ur, exi1));
              } else {
                exr0 = fmaf(tr, ur, fmaf(-ti, ui, exr0));
                exi0 = fmaf(tr, ui, fmaf(ti, ur, exi0));
              }
            }
            float dr = S[lane * 33 + a], di = S[lane * 33 + NP + a];   // T[a][a]
            float exr = exr0 + exr1, exi = exi0 + exi1;
#pragma unroll
            for (int o = NP / 2; o > 0; o >>= 1) {      // sums over the g block
              exr += __shfl_xor_sync(0xffffffffu, exr, o);
              exi += __shfl_xor_sync(0xffffffffu, exi, o);
              dr += __shfl_xor_sync(0xffffffffu, dr, o);
              di += __shfl_xor_sync(0xffffffffu, di, o);
            }
            const int w = ct * WPT + grp;
            if (a == 0 && g < X && w < Nw) trs[((int64_t)sp * Nw + w) * X + g] = make_float2(dr, di);
            float er = a == 0 ? -0.5f * exr : 0.f, ei = a == 0 ? -0.5f * exi : 0.f;
#pragma unroll
            for (int o = NP; o < 32; o <<= 1) {         // over the warp's g blocks
              er += __shfl_xor_sync(0xffffffffu, er, o);
              ei += __shfl_xor_sync(0xffffffffu, ei, o);
            }
            if (lane == 0) {
              rb[(quad * WPT + grp) * 2] = er;
              rb[(quad * WPT + grp) * 2 + 1] = ei;
            }
            __syncwarp();
            tmem_wait_ld_e();
          }
        } else if (lane == 0) {
          *s_fail = 1;
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(tempty0 + 8 * b);
        asm volatile("bar.sync 1, %0;" ::"n"(32 * EWARPS) : "memory");   // the epilogue warps
        if (*s_fail) { stop = true; break; }
        if (threadIdx.x < WPT)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            accr += rb[(q * WPT + threadIdx.x) * 2];
            acci += rb[(q * WPT + threadIdx.x) * 2 + 1];
          }
      }
      if (!stop && threadIdx.x < WPT) {
        const int w = ct * WPT + threadIdx.x, row = sp * NG + rg;
        part[(int64_t)(2 * row) * NwP + w] = accr;
        part[(int64_t)(2 * row + 1) * NwP + w] = acci;
      }
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

// (s, c) += (h + l) x, the product h x formed exactly (its rounding error recovered by an FMA,
// Dekker's two-product) and added to s by Knuth's two-sum; the intrinsics keep the compiler
// from contracting the error terms away
__device__ __forceinline__ void pair_acc(float& s, float& c, float h, float l, float x) {
  const float p = __fmul_rn(h, x);
  const float e = __fmaf_rn(h, x, -p);
  const float t = __fadd_rn(s, p);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, __fmaf_rn(l, x, e)));
}

// eloc[w] = sum_e htil[e] Theta_w[e] (FP32 pairs) + sum over row tiles of part for the first nw of
// the Nw walkers (one warp per walker;
// every sum in a fixed order, so repeated evaluations agree bit for bit).
// E_L per walker: the one-body term sum htil . Theta (FP64), the row tiles' partial two-body
// sums in a fixed order, and (spin-blocked layout) the Coulomb term 1/2 sum_g (sum_s tr T^s_g)^2
// from the traces trs ([2][Nw][X] complex); trs null: already in the partials.
__global__ void __launch_bounds__(256) k_energy_tc_reduce(const float* __restrict__ part, int RT, int NwP,
                                                          const float* __restrict__ th,
                                                          const float* __restrict__ hh,
                                                          const float* __restrict__ hl,
                                                          double* __restrict__ eloc, int Nw, int nw,
                                                          int NM, const float2* __restrict__ trs,
                                                          int X) {
  const int lane = threadIdx.x & 31, w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= nw) return;
  const int64_t plane = (int64_t)Nw * NM;
  // one-body term in FP32 pairs (GB300's FP64 pipe is thin): each product (hh + hl) theta
  // formed exactly up to the hl term (two-product by FMA) and added with a two-sum
  float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
  for (int e = lane; e < NM; e += 32) {
    const float h = __ldg(hh + e), l = __ldg(hl + e);
    const float tr = th[(int64_t)w * NM + e], ti = th[plane + (int64_t)w * NM + e];
    pair_acc(sr, cr, h, l, tr);
    pair_acc(si, ci, h, l, ti);
  }
  double r = (double)sr + (double)cr, i = (double)si + (double)ci;
  if (trs)
    for (int g = lane; g < X; g += 32) {
      const float2 u = trs[(int64_t)w * X + g], d = trs[((int64_t)Nw + w) * X + g];
      const double pr = (double)u.x + (double)d.x, pi = (double)u.y + (double)d.y;
      r += 0.5 * (pr * pr - pi * pi);
      i += pr * pi;
    }
  for (int t = lane; t < RT; t += 32) {
    r += (double)part[(int64_t)(2 * t) * NwP + w];
    i += (double)part[(int64_t)(2 * t + 1) * NwP + w];
  }
  for (int o = 16; o > 0; o >>= 1) {
    r += __shfl_xor_sync(0xffffffffu, r, o);
    i += __shfl_xor_sync(0xffffffffu, i, o);
  }
  if (lane == 0) {
    eloc[w] = r;
    eloc[Nw + w] = i;
  }
}

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

// x (FP64) as the FP32 pair hi + lo
__global__ void k_split_pair(const double* __restrict__ x, int n, float* __restrict__ hi,
                             float* __restrict__ lo) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const float h = (float)x[e];
    hi[e] = h;
    lo[e] = (float)(x[e] - (double)h);
  }
}

// spin-blocked form (M > 64): NPS = P2 rows per Cholesky vector and spin
template <int NPS>
cudaError_t launch_spin(const Ctx& c, const EnergyTc& et, int n_walkers, cudaStream_t s) {
  using Lay = ELayout<NPS>;
  const int NM = c.N * c.M, nw = n_walkers > 0 ? n_walkers : c.Nw;
  const int RTs = et.RT / 2, CTs = (c.Nw * 2 * NPS + EBN - 1) / EBN;
  k_energy_B_spin<<<grid_for((int64_t)2 * CTs * EBN * et.Kp), 256, 0, s>>>(
      c.theta32, c.Nw, c.N, c.M, c.n_up, NPS, et.Kp, CTs, nw, et.B->hi, et.B->lo);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int nparts = et.RT;
  if (NPS == 16 && et.Kp == 2 * EBK) {
    // Theta tile resident per (spin, column tile, row group) item, about 8 items per SM
    const int ng = std::max(1, std::min(RTs, (152 * 8 + 2 * CTs - 1) / (2 * CTs)));
    const int rg = (RTs + ng - 1) / ng;
    const int NG = (RTs + rg - 1) / rg;
    nparts = 2 * NG;
    const int grid = std::min(2 * CTs * NG, 152);
    k_energy_tc_spin2<16><<<grid, EPTHREADS, ES2Layout<16>::SMEM_BYTES, s>>>(
        et.A->map_hi, et.A->map_lo, et.B->map_hi, et.B->map_lo, RTs, CTs, rg, NG, et.part, et.NwP,
        c.d_tc_err, kEWaitNs, reinterpret_cast<float2*>(et.trs), c.X, c.Nw);
  } else {
    const int grid = std::min(2 * RTs * CTs, 152);
    k_energy_tc<NPS, true><<<grid, EPTHREADS, Lay::SMEM_BYTES, s>>>(
        et.A->map_hi, et.A->map_lo, et.B->map_hi, et.B->map_lo, et.Kp / EBK, RTs, CTs, et.part,
        et.NwP, c.d_tc_err, kEWaitNs, reinterpret_cast<float2*>(et.trs), c.X, c.Nw);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_energy_tc_reduce<<<(nw + 7) / 8, 256, 0, s>>>(et.part, nparts, et.NwP, c.theta32, et.hh, et.hl, c.eloc,
                                                  c.Nw, nw, NM, reinterpret_cast<const float2*>(et.trs),
                                                  c.X);
  return cudaGetLastError();
}

template <int NP>
cudaError_t launch_np(const Ctx& c, const EnergyTc& et, int n_walkers, cudaStream_t s) {
  using Lay = ELayout<NP>;
  const int NM = c.N * c.M, nw = n_walkers > 0 ? n_walkers : c.Nw;
  k_energy_B<<<grid_for((int64_t)nw * 2 * NP * et.Kp), 256, 0, s>>>(
      c.theta32, c.Nw, c.N, c.M, c.n_up, NP, et.Kp, et.B->hi, et.B->lo);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int ct = (nw * 2 * NP + EBN - 1) / EBN;
  int nparts = et.RT;
  if (et.Kp == EBK) {
    // B-resident form: about six (column tile, row group) items per SM
    const int ng = std::max(1, std::min(et.RT, (152 * 6 + ct - 1) / ct));
    const int rg = (et.RT + ng - 1) / ng;
    nparts = (et.RT + rg - 1) / rg;
    const int grid = std::min(ct * nparts, 152);
    k_energy_tc_bres<NP><<<grid, EBLayout<NP>::THREADS, EBLayout<NP>::SMEM_BYTES, s>>>(
        et.A->map_hi, et.A->map_lo, et.B->map_hi, et.B->map_lo, et.RT, ct, rg, nparts, et.part, et.NwP,
        c.d_tc_err, kEWaitNs);
  } else {
    const int grid = std::min(et.RT * ct, 152);
    k_energy_tc<NP, false><<<grid, EPTHREADS, Lay::SMEM_BYTES, s>>>(
        et.A->map_hi, et.A->map_lo, et.B->map_hi, et.B->map_lo, et.Kp / EBK, et.RT, ct, et.part,
        et.NwP, c.d_tc_err, kEWaitNs, nullptr, c.X, c.Nw);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_energy_tc_reduce<<<(nw + 7) / 8, 256, 0, s>>>(et.part, nparts, et.NwP, c.theta32, et.hh, et.hl, c.eloc,
                                                 c.Nw, nw, NM, nullptr, 0);
  return cudaGetLastError();
}

}  // namespace

int energy_tc_np(const Ctx& c) {
  const int m = std::max(c.n_up, c.N - c.n_up);
  int p2 = 4;
  while (p2 < m) p2 <<= 1;
  return p2 <= 16 ? 2 * p2 : 0;
}

cudaError_t prepare_energy_tc_kernels() {
  cudaError_t e = cudaFuncSetAttribute(k_energy_tc<8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       ELayout<8>::SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_energy_tc<16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             ELayout<16>::SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_energy_tc<32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             ELayout<32>::SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_energy_tc<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             ELayout<4>::SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_energy_tc<8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             ELayout<8>::SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_energy_tc<16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             ELayout<16>::SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_energy_tc_spin2<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             ES2Layout<16>::SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_energy_tc_bres<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             EBLayout<8>::SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_energy_tc_bres<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             EBLayout<16>::SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_energy_tc_bres<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             EBLayout<32>::SMEM_BYTES);
  return e;
}

// Operand buffers are allocated by the caller (sizes from energy_tc_sizes); this fills the
// A operand and encodes both tensor maps.
// M > 64 (more than one 64-wide k slice): the spin-blocked layout, rows of P2 = NP / 2 per
// Cholesky vector and spin, RT counting the row tiles of both spins
bool energy_tc_spin(const Ctx& c) { return pad64(c.M) > EBK; }

void energy_tc_sizes(const Ctx& c, int NP, int* rows_A, int* rows_B, int* Kp, int* RT, int* NwP) {
  *Kp = pad64(c.M);
  if (energy_tc_spin(c)) {
    const int P2 = NP / 2;
    const int RTs = (c.X * P2 + EBM - 1) / EBM, CTs = (c.Nw * 2 * P2 + EBN - 1) / EBN;
    *rows_A = 2 * RTs * EBM;
    *rows_B = 2 * CTs * EBN;
    *RT = 2 * RTs;
    *NwP = CTs * EBN / (2 * P2);
    return;
  }
  *rows_A = (c.X * NP + EBM - 1) / EBM * EBM;
  *rows_B = (c.Nw * 2 * NP + EBN - 1) / EBN * EBN;
  *RT = *rows_A / EBM;
  *NwP = *rows_B / (2 * NP);
}

cudaError_t energy_tc_init(const Ctx& c, EnergyTc& et, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(et.A->hi, 0, sizeof(__nv_bfloat16) * (size_t)et.A->rows * et.Kp, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(et.A->lo, 0, sizeof(__nv_bfloat16) * (size_t)et.A->rows * et.Kp, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(et.B->hi, 0, sizeof(__nv_bfloat16) * (size_t)et.B->rows * et.Kp, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(et.B->lo, 0, sizeof(__nv_bfloat16) * (size_t)et.B->rows * et.Kp, s);
  if (e != cudaSuccess) return e;
  if (energy_tc_spin(c))
    k_energy_A_spin<<<grid_for((int64_t)et.A->rows * et.Kp), 256, 0, s>>>(
        c.Ltil, c.X, c.N, c.M, c.n_up, et.NP / 2, et.Kp, et.RT / 2, et.A->hi, et.A->lo);
  else
    k_energy_A<<<grid_for((int64_t)c.X * et.NP * et.Kp), 256, 0, s>>>(c.Ltil, c.X, c.N, c.M, c.n_up,
                                                                     et.NP, et.Kp, et.A->hi, et.A->lo);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_split_pair<<<grid_for((int64_t)c.N * c.M), 256, 0, s>>>(c.htil, c.N * c.M, et.hh, et.hl);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = tc_make_operand(*et.A, et.A->hi, et.A->lo, et.A->rows, et.Kp, EBM)) != cudaSuccess) return e;
  return tc_make_operand(*et.B, et.B->hi, et.B->lo, et.B->rows, et.Kp, EBN / 2);
}

cudaError_t launch_energy_tc(const Ctx& c, cudaStream_t s, int n_walkers) {
  const EnergyTc& et = *c.etc;
  if (energy_tc_spin(c)) {
    switch (et.NP) {
      case 8: return launch_spin<4>(c, et, n_walkers, s);
      case 16: return launch_spin<8>(c, et, n_walkers, s);
      case 32: return launch_spin<16>(c, et, n_walkers, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (et.NP) {
    case 8: return launch_np<8>(c, et, n_walkers, s);
    case 16: return launch_np<16>(c, et, n_walkers, s);
    case 32: return launch_np<32>(c, et, n_walkers, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace afq
