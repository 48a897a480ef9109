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

constexpr int EBM = 128, EBN = 256, EBK = 64, ETHREADS = 128;
constexpr uint64_t kEWaitNs = 2000000000ull;

__host__ __device__ constexpr int cols_per_group(int NP) { return 2 * NP > 32 ? 2 * NP : 32; }

// One stage (A and B of one 64-wide k slice); the epilogue reuses it as its staging buffer
// once every MMA has completed, so a CTA needs ~97 KB and two CTAs (2 x 256 TMEM columns)
// share an SM.
template <int NP>
struct ELayout {
  static constexpr int A_BYTES = EBM * EBK * 2;                 // one of hi / lo
  static constexpr int B_BYTES = EBN * EBK * 2;
  static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int CW = cols_per_group(NP);                 // TMEM columns staged per step
  static constexpr int STG_BYTES = 4 * 32 * (CW + 1) * 4;       // per warp 32 rows x (CW + 1)
  static constexpr int WPT = EBN / (2 * NP);                    // walkers per tile
  static constexpr int RED_OFFSET = STAGE_BYTES;
  static constexpr int RED_BYTES = 4 * WPT * 2 * 4;
  static constexpr int BAR_OFFSET = (RED_OFFSET + RED_BYTES + 7) & ~7;
  static constexpr int SMEM_BYTES = BAR_OFFSET + 64 + 1024;     // 3 barriers, TMEM slot, alignment
  static_assert(STG_BYTES <= STAGE_BYTES, "staging must fit in the operand stage");
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

// ---------------------------------------------------------------------------
// One 128 x 256 tile of T per CTA (4 warps): warp 0 / lane 0 issues the TMA loads of the
// k slices (A hi/lo: one 128-row box each; B hi/lo: two 128-row boxes each) into the single
// stage, warp 1 / lane 0 issues 4 x 3 tcgen05.mma (K = 16, N = 256) per slice into TMEM and
// commits; all warps then run the epilogue on their 32 TMEM lanes (= rows (g, a)).
// part[(tile_row * 2 + re/im) * NwP + w] = sum over the tile's g of E2(g, w).
// Every mbarrier wait is bounded; on expiry *err is set, the CTA drains what it issued,
// frees its TMEM and writes zeros.
// ---------------------------------------------------------------------------
template <int NP>
__global__ void __launch_bounds__(ETHREADS, 1)
    k_energy_tc(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                int nkb, float* __restrict__ part, int NwP, int* err, uint64_t wait_ns) {
  using Lay = ELayout<NP>;
  constexpr int CW = Lay::CW, WPT = Lay::WPT, P2 = NP / 2, WPG = CW / (2 * NP);
  extern __shared__ uint8_t esm_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(esm_raw) + 1023) &
                                             ~uintptr_t(1023));
  float* red = reinterpret_cast<float*>(smem + Lay::RED_OFFSET);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Lay::BAR_OFFSET);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3);
  const uint32_t full = smem_u32(bars), empty = smem_u32(bars + 1), done = smem_u32(bars + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * EBM, n0 = blockIdx.y * EBN;

  for (int e = threadIdx.x; e < 4 * WPT * 2; e += ETHREADS) red[e] = 0.f;
  if (threadIdx.x == 0) {
    mbar_init(full, 1);
    mbar_init(empty, 1);
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"((uint32_t)EBN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t st = smem_u32(smem);

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: slice kb reuses the stage after the MMAs of slice kb-1 released it ----
    int issued = 0;
    for (int kb = 0; kb < nkb; ++kb) {
      if (kb > 0 && !mbar_wait(empty, (kb - 1) & 1, err, wait_ns)) break;
      mbar_expect_tx(full, Lay::STAGE_BYTES);
      const int kx = kb * EBK;
      tma_load_2d(st, &tmAh, full, kx, m0);
      tma_load_2d(st + Lay::A_BYTES, &tmAl, full, kx, m0);
      const uint32_t bh = st + 2 * Lay::A_BYTES, bl = bh + Lay::B_BYTES;
      tma_load_2d(bh, &tmBh, full, kx, n0);
      tma_load_2d(bh + Lay::B_BYTES / 2, &tmBh, full, kx, n0 + EBN / 2);
      tma_load_2d(bl, &tmBl, full, kx, n0);
      tma_load_2d(bl + Lay::B_BYTES / 2, &tmBl, full, kx, n0 + EBN / 2);
      issued = kb + 1;
    }
    // drain: the last issued slice must have landed before the CTA may exit
    if (issued > 0) mbar_wait(full, (issued - 1) & 1, err, wait_ns);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    const uint32_t idesc = idesc_bf16<EBN>();
    for (int kb = 0; kb < nkb; ++kb) {
      if (!mbar_wait(full, kb & 1, err, wait_ns)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t ah = sw128_desc(st), al = sw128_desc(st + Lay::A_BYTES);
      const uint64_t bh = sw128_desc(st + 2 * Lay::A_BYTES);
      const uint64_t bl = sw128_desc(st + 2 * Lay::A_BYTES + Lay::B_BYTES);
#pragma unroll
      for (int kk = 0; kk < EBK / 16; ++kk) {
        const uint64_t dk = (uint64_t)((kk * 32) >> 4);   // 16 bf16 = 32 bytes inside the atom
        mma_bf16(tmem, ah + dk, bh + dk, idesc, (kb | kk) != 0);
        mma_bf16(tmem, ah + dk, bl + dk, idesc, 1u);
        mma_bf16(tmem, al + dk, bh + dk, idesc, 1u);
      }
      mma_commit(empty);
    }
    mma_commit(done);   // also on an early exit: arrives once the issued MMAs are complete
  }
  __syncwarp();

  // ---- epilogue ----
  const bool ok = mbar_wait(done, 0, err, 2 * wait_ns);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncwarp();
  // the operand stage is free once every MMA has completed: stage TMEM rows there
  float* S = reinterpret_cast<float*>(smem) + warp * 32 * (CW + 1);
  const int a = lane % NP, gl = lane / NP, s0 = a < P2 ? 0 : P2;
  if (__all_sync(0xffffffffu, ok && *(volatile int*)err == 0)) {
    for (int grp = 0; grp < EBN / CW; ++grp) {
#pragma unroll
      for (int h = 0; h < CW / 32; ++h) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(grp * CW + 32 * h), v);
#pragma unroll
        for (int j = 0; j < 32; ++j) S[lane * (CW + 1) + 32 * h + j] = __uint_as_float(v[j]);
      }
      __syncwarp();
#pragma unroll
      for (int wi = 0; wi < WPG; ++wi) {
        const int cb = wi * 2 * NP;
        const float* rowp = S + lane * (CW + 1) + cb;               // T[a][.] (re, then im)
        const float* colp = S + gl * NP * (CW + 1) + cb + a;        // T[.][a]
        float exr = 0.f, exi = 0.f;
#pragma unroll
        for (int j = 0; j < P2; ++j) {
          const int b = s0 + j;
          const float tr = rowp[b], ti = rowp[NP + b];
          const float ur = colp[b * (CW + 1)], ui = colp[b * (CW + 1) + NP];
          exr = fmaf(tr, ur, fmaf(-ti, ui, exr));
          exi = fmaf(tr, ui, fmaf(ti, ur, exi));
        }
        float dr = rowp[a], di = rowp[NP + a];
#pragma unroll
        for (int o = NP / 2; o > 0; o >>= 1) {                     // sums over the g block
          exr += __shfl_xor_sync(0xffffffffu, exr, o);
          exi += __shfl_xor_sync(0xffffffffu, exi, o);
          dr += __shfl_xor_sync(0xffffffffu, dr, o);
          di += __shfl_xor_sync(0xffffffffu, di, o);
        }
        float er = a == 0 ? 0.5f * (dr * dr - di * di - exr) : 0.f;
        float ei = a == 0 ? 0.5f * (2.f * dr * di - exi) : 0.f;
#pragma unroll
        for (int o = NP; o < 32; o <<= 1) {                        // over the warp's g blocks
          er += __shfl_xor_sync(0xffffffffu, er, o);
          ei += __shfl_xor_sync(0xffffffffu, ei, o);
        }
        if (lane == 0) {
          red[(warp * WPT + grp * WPG + wi) * 2] = er;
          red[(warp * WPT + grp * WPG + wi) * 2 + 1] = ei;
        }
      }
      __syncwarp();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < WPT) {
    const int t = threadIdx.x, w = blockIdx.y * WPT + t;
    float sr = 0.f, si = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      sr += red[(q * WPT + t) * 2];
      si += red[(q * WPT + t) * 2 + 1];
    }
    part[(int64_t)(2 * blockIdx.x) * NwP + w] = sr;
    part[(int64_t)(2 * blockIdx.x + 1) * NwP + w] = si;
  }
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)EBN)
                 : "memory");
}

// eloc[w] = sum_e htil[e] Theta_w[e] (FP64) + sum over row tiles of part for the first nw of
// the Nw walkers (one warp per walker;
// every sum in a fixed order, so repeated evaluations agree bit for bit).
__global__ void __launch_bounds__(256) k_energy_tc_reduce(const float* __restrict__ part, int RT, int NwP,
                                                          const float* __restrict__ th,
                                                          const double* __restrict__ htil,
                                                          double* __restrict__ eloc, int Nw, int nw,
                                                          int NM) {
  const int lane = threadIdx.x & 31, w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= nw) return;
  const int64_t plane = (int64_t)Nw * NM;
  double r = 0.0, i = 0.0;
  for (int e = lane; e < NM; e += 32) {
    const double h = __ldg(htil + e);
    r = fma(h, (double)th[(int64_t)w * NM + e], r);
    i = fma(h, (double)th[plane + (int64_t)w * NM + e], i);
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

template <int NP>
cudaError_t launch_np(const Ctx& c, const EnergyTc& et, int n_walkers, cudaStream_t s) {
  using Lay = ELayout<NP>;
  const int NM = c.N * c.M, nw = n_walkers > 0 ? n_walkers : c.Nw;
  k_energy_B<<<grid_for((int64_t)nw * 2 * NP * et.Kp), 256, 0, s>>>(
      c.theta32, c.Nw, c.N, c.M, c.n_up, NP, et.Kp, et.B->hi, et.B->lo);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int ct = (nw * 2 * NP + EBN - 1) / EBN;
  dim3 grid(et.RT, ct);
  k_energy_tc<NP><<<grid, ETHREADS, Lay::SMEM_BYTES, s>>>(et.A->map_hi, et.A->map_lo, et.B->map_hi,
                                                         et.B->map_lo, et.Kp / EBK, et.part, et.NwP,
                                                         c.d_tc_err, kEWaitNs);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_energy_tc_reduce<<<(nw + 7) / 8, 256, 0, s>>>(et.part, et.RT, et.NwP, c.theta32, c.htil, c.eloc,
                                                 c.Nw, nw, NM);
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
  cudaError_t e = cudaFuncSetAttribute(k_energy_tc<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       ELayout<8>::SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_energy_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             ELayout<16>::SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_energy_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             ELayout<32>::SMEM_BYTES);
  return e;
}

// Operand buffers are allocated by the caller (sizes from energy_tc_sizes); this fills the
// A operand and encodes both tensor maps.
void energy_tc_sizes(const Ctx& c, int NP, int* rows_A, int* rows_B, int* Kp, int* RT, int* NwP) {
  *Kp = pad64(c.M);
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
  k_energy_A<<<grid_for((int64_t)c.X * et.NP * et.Kp), 256, 0, s>>>(c.Ltil, c.X, c.N, c.M, c.n_up, et.NP,
                                                                   et.Kp, et.A->hi, et.A->lo);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = tc_make_operand(*et.A, et.A->hi, et.A->lo, et.A->rows, et.Kp, EBM)) != cudaSuccess) return e;
  return tc_make_operand(*et.B, et.B->hi, et.B->lo, et.B->rows, et.Kp, EBN / 2);
}

cudaError_t launch_energy_tc(const Ctx& c, cudaStream_t s, int n_walkers) {
  const EnergyTc& et = *c.etc;
  switch (et.NP) {
    case 8: return launch_np<8>(c, et, n_walkers, s);
    case 16: return launch_np<16>(c, et, n_walkers, s);
    case 32: return launch_np<32>(c, et, n_walkers, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace afq
