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

#include "device_util.cuh"
#include "internal.h"
#include "tc_device.cuh"

namespace afq {
namespace {

using namespace tc;

constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int kTile = 128 * 64 * 2;       // one 128-row x 64-K bf16 tile, 128-byte swizzle
constexpr int kMaxStages = 12;
constexpr int kXu = 4;                    // staged-X elements per epilogue thread and round

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

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// L2 prefetch hint over the 16-byte-aligned interior of [p, p + bytes) (the bulk prefetch needs a
// 16-byte-aligned address and size)
__device__ __forceinline__ void prefetch_l2(const void* p, uint64_t bytes) {
  const uint64_t a = reinterpret_cast<uint64_t>(p);
  const uint64_t lo = (a + 15) & ~uint64_t(15), hi = (a + bytes) & ~uint64_t(15);
  if (hi > lo)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((uint32_t)(hi - lo))
                 : "memory");
}

// One 16-lane x 16-column block of 32-bit TMEM cells in the mma fragment layout: thread t holds
// lanes t/4 (v[0,1], v[4,5]) and 8 + t/4 (v[2,3], v[6,7]), columns 2 (t%4) + {0, 1} (v[0..3])
// and 8 + 2 (t%4) + {0, 1} (v[4..7]).
__device__ __forceinline__ void tmem_ld_frag(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.16x256b.x2.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                 "=r"(v[7])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_st_frag(uint32_t taddr, const uint32_t (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.16x256b.x2.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(
                   taddr),
               "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}

// Transposed 8x8 stores of 16-bit pairs: register j of thread t holds row t/4, columns
// 2 (t%4) + {0, 1} of matrix j; row k of matrix j (its column k) goes to the 16 bytes at the
// address thread 8 j + k supplies.
__device__ __forceinline__ void stsm_x4_t(uint32_t addr, const uint32_t (&r)[4]) {
  asm volatile("stmatrix.sync.aligned.m8n8.x4.trans.shared.b16 [%0], {%1, %2, %3, %4};" ::"r"(addr),
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3])
               : "memory");
}

__device__ __forceinline__ void stsm_x2_t(uint32_t addr, uint32_t r0, uint32_t r1) {
  asm volatile("stmatrix.sync.aligned.m8n8.x2.trans.shared.b16 [%0], {%1, %2};" ::"r"(addr), "r"(r0),
               "r"(r1)
               : "memory");
}

__device__ __forceinline__ uint32_t elect_one() {
  uint32_t p;
  asm volatile("{\n\t.reg .pred P;\n\telect.sync _|P, 0xffffffff;\n\tselp.u32 %0, 1, 0, P;\n\t}"
               : "=r"(p));
  return p;
}

// x = hi + lo for a pair of floats (a in the low half): both halves as packed BF16 pairs
__device__ __forceinline__ void split_pair(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - __low2float(h), b - __high2float(h));
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// One product round with every A plane in tensor memory (plane u, K block kb at abase + 32 (u KB
// + kb)): NPL = 4 for a Taylor term (A_re hi, lo, A_im hi, lo), 2 for a one-body half step (E - I
// hi, lo).  B descriptors dbh / dbl address the term operand; A_re and E - I take rows Np..3Np
// (offset np16), A_im rows 0..2Np.  The hi planes take two MMAs per 16-wide K step (x B hi,
// x B lo), the lo planes one; the last K block stops after nks_last steps.
template <int KB, int NPL>
__device__ __forceinline__ void mma_round_tmem(uint32_t d, uint32_t abase, uint64_t dbh, uint64_t dbl,
                                               uint32_t bkb16, uint32_t np16, uint32_t idesc,
                                               int nks_last) {
#pragma unroll
  for (int kb = 0; kb < KB; ++kb)
#pragma unroll
    for (int u = 0; u < NPL; ++u) {
      const uint32_t ta = abase + (uint32_t)(32 * (u * KB + kb));
      const uint64_t roff = (uint64_t)(kb * bkb16 + (u >= 2 ? 0u : np16));
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        if (kb == KB - 1 && ks >= nks_last) break;
        const uint64_t dk = roff + (uint64_t)(2 * ks);
        mma_bf16_ta(d, ta + (uint32_t)(8 * ks), dbh + dk, idesc, (kb | u | ks) != 0 ? 1u : 0u);
        if ((u & 1) == 0) mma_bf16_ta(d, ta + (uint32_t)(8 * ks), dbl + dk, idesc, 1u);
      }
    }
}

// Static shape of one launch (host-computed).
struct TclShape {
  const __nv_bfloat16 *ahi, *alo;   // V_HS split planes [2][Nw][M][Mp] (L2 prefetch of the next walker)
  int Mp;                // elements per orbital row of the split planes
  int M, N, Np, n2;      // orbitals, occupied columns, N rounded up to 8, MMA N = 2 Np
  int MT, KB;            // 128-row tiles of orbitals, 64-wide K blocks
  int nst;               // ring stages
  int resident;          // 1: A of a walker held in tensor memory for all its Taylor rounds,
                         // staged through a shared-memory region the producer fills ahead
  int ares_off;          // shared staging of A: 4 KB tiles (A_re hi, lo, A_im hi, lo per K block)
  int acol;              // resident form: TMEM column of A (plane P, K block kb at acol + 32 (P KB + kb))
  int eres, ecol;        // 1: e^{-dt K/2} - I also in tensor memory (hi, lo planes from ecol), loaded
                         // once per CTA; the one-body rounds then need no ring
  int bkb;               // bytes of one K block of the term operand (3 Np rows x 128 bytes)
  int dcol;              // TMEM column stride between tiles (D and S regions)
  uint32_t tcols;        // TMEM columns allocated
  int order, Nw;
  int xs, xs_ld;         // 1: the next walker's X (FP32, rows c of xs_ld floats) staged in the ring
                         // region during the current walker's rounds (resident form with E in
                         // tensor memory, which leaves the ring unused)
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
  const uint32_t afull = smem_u32(bars + 2 * kMaxStages + 3), acopied = smem_u32(bars + 2 * kMaxStages + 4);
  const uint32_t xfull = smem_u32(bars + 2 * kMaxStages + 5), xread = smem_u32(bars + 2 * kMaxStages + 6);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kMaxStages + 7);
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
    mbar_init(acopied, 32 * EPI);
    mbar_init(xfull, 32 * EPI);
    mbar_init(xread, 32 * EPI);
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
      if (sh.eres) {
        // e^{-dt K/2} - I through the staging region into tensor memory, once per CTA
        mbar_expect_tx(afull, 2 * sh.KB * kTile);
        for (int kb = 0; kb < sh.KB; ++kb)
          for (int u = 0; u < 2; ++u)
            tma_load_2d(smem_u32(smem + sh.ares_off + (kb * 4 + u) * kTile), u ? &tmElo : &tmEhi, afull,
                        kb * 64, 0);
        ++aw;
      }
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
          if (sh.resident && q == 0) {
            // this walker's A into the staging region once the epilogue has copied the previous
            // walker's A to tensor memory (acopied), all tiles on one barrier
            if (aw > 0 && !mbar_wait(acopied, (aw - 1) & 1, err, wait_ns)) {
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
          if (sh.resident && (taylor || sh.eres)) continue;
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
    // ---- MMA issuer: the whole warp follows the loop, so every operand address is warp-uniform,
    // and one elected lane issues; lane 0 polls the barriers and broadcasts the outcome ----
    const uint32_t idesc = idesc_n(sh.n2);
    const uint32_t bhi = smem_u32(smem + sh.bhi_off), blo = smem_u32(smem + sh.blo_off);
    const uint64_t dbh = sw128_desc(bhi), dbl = sw128_desc(blo);
    const uint32_t bkb16 = (uint32_t)(sh.bkb >> 4), np16 = (uint32_t)(sh.Np * 8);
    const int nks_last = min(4, (sh.M - 64 * (sh.KB - 1) + 15) / 16);
    int g = 0, rq = 0;
    bool ok = true;
    auto wait_all = [&](uint32_t bar, int parity) {
      int okw = 1;
      if (lane == 0) okw = !*abort_flag && mbar_wait(bar, parity, err, wait_ns);
      okw = __shfl_sync(0xffffffffu, okw, 0);
      if (!okw && lane == 0) fail();
      return okw != 0;
    };
    for (int w = blockIdx.x; w < sh.Nw && ok; w += gridDim.x) {
      if (alive && !alive[w]) continue;
      for (int q = 0; q < rounds && ok; ++q, ++rq) {
        const bool taylor = q >= 1 && q <= sh.order;
        if (!wait_all(bready, rq & 1)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (sh.resident && (taylor || sh.eres)) {
          // every A plane in tensor memory (one tile row, MT = 1)
          if (elect_one()) {
            if (sh.KB == 2) {
              if (taylor)
                mma_round_tmem<2, 4>(tmem, tmem + (uint32_t)sh.acol, dbh, dbl, bkb16, np16, idesc, nks_last);
              else
                mma_round_tmem<2, 2>(tmem, tmem + (uint32_t)sh.ecol, dbh, dbl, bkb16, np16, idesc, nks_last);
            } else {
              if (taylor)
                mma_round_tmem<1, 4>(tmem, tmem + (uint32_t)sh.acol, dbh, dbl, bkb16, np16, idesc, nks_last);
              else
                mma_round_tmem<1, 2>(tmem, tmem + (uint32_t)sh.ecol, dbh, dbl, bkb16, np16, idesc, nks_last);
            }
            mma_commit(dfull);
          }
          __syncwarp();
          continue;
        }
        for (int t = 0; t < sh.MT && ok; ++t) {
          const uint32_t d = tmem + (uint32_t)(t * sh.dcol);
          for (int kb = 0; kb < sh.KB && ok; ++kb) {
            const int nks = kb == sh.KB - 1 ? nks_last : 4;   // K steps holding orbitals
            for (int u = 0; u < (taylor ? 4 : 2); ++u, ++g) {
              const int st = g % sh.nst, use = g / sh.nst;
              if (!wait_all(full0 + 8 * st, use & 1)) { ok = false; break; }
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
              if (elect_one()) {
                const uint64_t a = sw128_desc(smem_u32(smem + sh.ring_off + st * kTile));
                // A_im (u >= 2) takes rows 0..2Np of the term operand, A_re and E - I rows Np..3Np
                const uint64_t roff = (uint64_t)(kb * bkb16 + ((taylor && u >= 2) ? 0u : np16));
                const bool hi = (u & 1) == 0;
                for (int ks = 0; ks < nks; ++ks) {
                  const uint64_t dk = roff + (uint64_t)(2 * ks);   // 16 bf16 = 32 bytes along K
                  mma_bf16(d, a + (uint64_t)(2 * ks), dbh + dk, idesc, (kb | u | ks) != 0 ? 1u : 0u);
                  if (hi) mma_bf16(d, a + (uint64_t)(2 * ks), dbl + dk, idesc, 1u);
                }
                mma_commit(empty0 + 8 * st);
              }
              __syncwarp();
            }
          }
        }
        if (ok) {
          if (elect_one()) mma_commit(dfull);
          __syncwarp();
        }
      }
    }
    if (elect_one()) mma_commit(done);   // arrives once every issued MMA has completed
    __syncwarp();
  } else {
    // ---- epilogue: warp w owns TMEM lanes 32 (w % 4) .. + 31 as two 16-lane slabs, read and
    // written in the mma fragment layout; with 8 epilogue warps two share each lane quadrant and
    // take alternate 16-column groups.  The term operand is written by transposed 8x8 stores:
    // one 16-byte row chunk holds 8 consecutive orbitals of one operand row ----
    const int qd = warp & 3, r = 32 * qd + lane;
    const int half = EPI == 8 ? (warp - 2) >> 2 : 0, cstep = EPI == 8 ? 32 : 16;
    const uint32_t lanes = (uint32_t)(32 * qd) << 16;
    const uint32_t bhi_s = smem_u32(smem + sh.bhi_off), blo_s = smem_u32(smem + sh.blo_off);
    const uint32_t sreg = (uint32_t)(sh.MT * sh.dcol);   // S region after the D columns
    const int jj = lane >> 3, kk = lane & 7, fr = lane >> 2, fc = 2 * (lane & 3);
    // fragment element j: lane offset fr (+ 8), column offset fc (+ 1) (+ 8)
    auto lane_of = [&](int j) { return fr + ((j & 2) ? 8 : 0); };
    auto col_of = [&](int j) { return fc + (j & 1) + ((j & 4) ? 8 : 0); };
    // shared address of the row chunk (operand row R, orbitals i0 .. i0 + 7) of one 8x8 store
    auto chunk = [&](uint32_t buf, int R, int i0) {
      return buf + (uint32_t)((i0 >> 6) * sh.bkb + R * 128 + ((((i0 & 63) >> 3) ^ (R & 7)) << 4));
    };
    // the block's values (orbitals i0b .., columns c0 ..) into operand rows Np + c, and with neg,
    // -value into rows c - Np for the imaginary columns c >= Np
    auto put_block = [&](const float (&v)[8], int i0b, int c0, bool neg) {
      uint32_t h[4], l[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) split_pair(v[2 * j], v[2 * j + 1], h[j], l[j]);
      // matrix jj: orbitals i0b + 8 (jj & 1) .., columns c0 + 8 (jj >> 1) ..; this lane: row kk
      const int i0 = i0b + 8 * (jj & 1), c = c0 + 8 * (jj >> 1) + kk;
      stsm_x4_t(chunk(bhi_s, sh.Np + c, i0), h);
      stsm_x4_t(chunk(blo_s, sh.Np + c, i0), l);
      if (!neg || c0 + 8 < sh.Np) return;   // no imaginary column in the group
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        h[j] ^= 0x80008000u;
        l[j] ^= 0x80008000u;
      }
      if (c0 >= sh.Np) {
        stsm_x4_t(chunk(bhi_s, c - sh.Np, i0), h);
        stsm_x4_t(chunk(blo_s, c - sh.Np, i0), l);
      } else {
        // only the second 8-column block is imaginary: matrices 2, 3 (lanes 0..15 give rows)
        const int cn = c0 + 8 + kk - sh.Np;
        stsm_x2_t(chunk(bhi_s, cn, i0), h[2], h[3]);
        stsm_x2_t(chunk(blo_s, cn, i0), l[2], l[3]);
      }
    };
    int rq = 0, jw = 0;
    bool ok = true;
    // resident A: the staging tiles into tensor memory; lane r takes row r of every tile (16-byte
    // chunks in the 128-byte swizzle), the two warps of a lane quadrant take planes
    // {2 half, 2 half + 1} of the first np planes, from TMEM column col0
    auto copy_planes = [&](int np, int col0) {
      const bool okw = !*abort_flag && mbar_wait(afull, jw & 1, err, wait_ns);
      if (!__all_sync(0xffffffffu, okw)) { fail(); return false; }
      for (int u = 2 * half; u < 2 * half + 2 && u < np; ++u)
        for (int kb = 0; kb < sh.KB; ++kb) {
          const uint4* row = reinterpret_cast<const uint4*>(smem + sh.ares_off + (kb * 4 + u) * kTile + r * 128);
          uint32_t v[32];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const uint4 c = row[j ^ (r & 7)];
            v[4 * j] = c.x; v[4 * j + 1] = c.y; v[4 * j + 2] = c.z; v[4 * j + 3] = c.w;
          }
          const uint32_t ta = tmem + lanes + (uint32_t)(col0 + 32 * (u * sh.KB + kb));
          tmem_st16(ta, *reinterpret_cast<const uint32_t(*)[16]>(v));
          tmem_st16(ta + 16, *reinterpret_cast<const uint32_t(*)[16]>(v + 16));
        }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      mbar_arrive(acopied);   // the staging region may take the next tiles
      ++jw;
      return true;
    };
    // this warp's (tile, slab, 16-column group) items: item it -> tile it / (2 ngh), slab
    // (it % 2 ngh) / ngh, columns 16 half + (it % ngh) cstep
    const int ngh = (sh.n2 - 16 * half + cstep - 1) / cstep;
    const int nitems = sh.MT * 2 * ngh;
    if (sh.eres && !copy_planes(2, sh.ecol)) ok = false;
    // staged X: element e of a walker is column c = e / M, orbital i = e % M (FP32); thread t of
    // the epilogue takes e = t + 32 EPI (q + rounds u) in round q, so a walker's X is loaded
    // during the previous walker's rounds, each load issued before the round's wait
    float* xst = reinterpret_cast<float*>(smem + sh.ring_off);
    const int et = threadIdx.x - 64, nte = 32 * EPI, nx = sh.n2 * sh.M;
    const int xu = (nx + nte * rounds - 1) / (nte * rounds);     // elements per thread and round
    const int xdc = nte / sh.M, xdi = nte - (nte / sh.M) * sh.M;
    auto x_elem = [&](int wn, int e) -> double {
      const int c = e / sh.M, i = e - c * sh.M, b = c < sh.Np ? c : c - sh.Np;
      return b < sh.N ? phi_in[(c < sh.Np ? 0 : plane) + ((int64_t)wn * sh.N + b) * sh.M + i] : 0.0;
    };
    auto x_put = [&](int e, double v) {
      const int c = e / sh.M, i = e - c * sh.M;
      xst[c * sh.xs_ld + i] = f64_to_f32_rn(v);
    };
    auto next_live = [&](int w) {
      int wn = w + (int)gridDim.x;
      while (wn < sh.Nw && alive && !alive[wn]) wn += (int)gridDim.x;
      return wn;
    };
    if (sh.xs && ok) {
      int w0 = blockIdx.x;
      while (w0 < sh.Nw && alive && !alive[w0]) w0 += (int)gridDim.x;
      if (w0 < sh.Nw)
        for (int e0 = et; e0 < nx; e0 += 4 * nte) {
          double v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) v[u] = e0 + u * nte < nx ? x_elem(w0, e0 + u * nte) : 0.0;
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (e0 + u * nte < nx) x_put(e0 + u * nte, v[u]);
        }
      mbar_arrive(xfull);
    }
    int kx = 0;   // live walkers of this CTA so far
    for (int w = blockIdx.x; w < sh.Nw && ok; w += gridDim.x) {
      if (alive && !alive[w]) continue;
      const int wn = sh.xs ? next_live(w) : sh.Nw;
      const int kw = kx++;
      // element cursor of this thread's share of the next walker's X: e = et + nte j,
      // (column, orbital) = divmod(e, M), advanced by (xdc, xdi) = divmod(nte, M)
      int xe = et, xc = et / sh.M, xi = et - (et / sh.M) * sh.M;
      if (sh.xs) {
        // this walker's X, staged by every epilogue thread, is complete
        const bool okx = !*abort_flag && mbar_wait(xfull, kw & 1, err, wait_ns);
        if (!__all_sync(0xffffffffu, okx)) { fail(); ok = false; break; }
        if (!copy_planes(4, sh.acol)) { ok = false; break; }
        for (int it = 0; it < nitems; ++it) {
          const int t = it / (2 * ngh), sl = (it % (2 * ngh)) / ngh;
          const int c0 = 16 * half + (it % ngh) * cstep, i0b = 128 * t + 32 * qd + 16 * sl;
          const uint32_t tl = tmem + ((uint32_t)(32 * qd + 16 * sl) << 16);
          float x[8];
          uint32_t v[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int i = i0b + lane_of(j), c = c0 + col_of(j);
            x[j] = i < sh.M ? xst[c * sh.xs_ld + i] : 0.f;
            v[j] = __float_as_uint(x[j]);
          }
          tmem_st_frag(tl + sreg + (uint32_t)(t * sh.dcol + c0), v);
          if (i0b < 64 * sh.KB) put_block(x, i0b, c0, false);
        }
        mbar_arrive(xread);   // the staged X may take the next walker's once all have read it
      } else
      // S = X (this walker's columns) and the operand [X_re; X_im] for the first one-body round.
      // The (tile, slab, column group) items of this warp go in batches of 4: every load of a
      // batch is issued first, so the walker pays one memory latency per batch, and the first
      // batch's loads are in flight while A moves into tensor memory.
      for (int b0 = 0; b0 == 0 || b0 < nitems; b0 += 4) {   // one pass at least: the A copy
        double xv[4][8];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int it = b0 + u, t = it / (2 * ngh), sl = (it % (2 * ngh)) / ngh;
          const int c0 = 16 * half + (it % ngh) * cstep, i0b = 128 * t + 32 * qd + 16 * sl;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int i = i0b + lane_of(j), c = c0 + col_of(j), b = c < sh.Np ? c : c - sh.Np;
            xv[u][j] = (it < nitems && i < sh.M && b < sh.N)
                           ? phi_in[(c < sh.Np ? 0 : plane) + ((int64_t)w * sh.N + b) * sh.M + i]
                           : 0.0;
          }
        }
        if (b0 == 0 && sh.resident && !copy_planes(4, sh.acol)) { ok = false; break; }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int it = b0 + u, t = it / (2 * ngh), sl = (it % (2 * ngh)) / ngh;
          const int c0 = 16 * half + (it % ngh) * cstep, i0b = 128 * t + 32 * qd + 16 * sl;
          if (it >= nitems) break;
          const uint32_t tl = tmem + ((uint32_t)(32 * qd + 16 * sl) << 16);
          float x[8];
          uint32_t v[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            x[j] = f64_to_f32_rn(xv[u][j]);
            v[j] = __float_as_uint(x[j]);
          }
          tmem_st_frag(tl + sreg + (uint32_t)(t * sh.dcol + c0), v);
          if (i0b < 64 * sh.KB) put_block(x, i0b, c0, false);
        }
      }
      if (!ok) break;
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(bready);
      for (int q = 0; q < rounds && ok; ++q, ++rq) {
        const bool last = q == rounds - 1;
        // this round's share of the next walker's X: loaded now, staged after the round's
        // results are handed to the MMA warp, so the loads have the MMAs and the round's
        // epilogue to land
        double xp[kXu];
        int xo[kXu];
        const bool pre = sh.xs && wn < sh.Nw;
        if (pre)
#pragma unroll
          for (int u = 0; u < kXu; ++u) {
            const bool v = u < xu && xe < nx;
            const int b = xc < sh.Np ? xc : xc - sh.Np;
            xp[u] = v && b < sh.N
                        ? phi_in[(xc < sh.Np ? 0 : plane) + ((int64_t)wn * sh.N + b) * sh.M + xi]
                        : 0.0;
            xo[u] = v ? xc * sh.xs_ld + xi : -1;
            if (v) {   // the thread's next element: e + nte
              xe += nte;
              xc += xdc;
              xi += xdi;
              if (xi >= sh.M) { xi -= sh.M; ++xc; }
            }
          }
        bool okw = !*abort_flag && mbar_wait(dfull, rq & 1, err, wait_ns);
        if (pre && q == 0) okw = okw && !*abort_flag && mbar_wait(xread, kw & 1, err, wait_ns);
        if (!__all_sync(0xffffffffu, okw)) { fail(); ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const float inv = (q >= 1 && q <= sh.order) ? 1.f / (float)q : 1.f;
        for (int t = 0; t < sh.MT; ++t)
          for (int sl = 0; sl < 2; ++sl) {
            const int i0b = 128 * t + 32 * qd + 16 * sl;
            const bool in_b = i0b < 64 * sh.KB;
            const uint32_t tl = tmem + ((uint32_t)(32 * qd + 16 * sl) << 16);
            for (int c0 = 16 * half; c0 < sh.n2; c0 += cstep) {
              uint32_t dv[8], sv[8];
              tmem_ld_frag(tl + (uint32_t)(t * sh.dcol + c0), dv);
              tmem_ld_frag(tl + sreg + (uint32_t)(t * sh.dcol + c0), sv);
              tmem_wait_ld();
              float x[8];
              if (q == 0) {
                // T_0 = X + (E - I) X: S = T_0, operand = T_0
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  x[j] = __uint_as_float(sv[j]) + __uint_as_float(dv[j]);
                  sv[j] = __float_as_uint(x[j]);
                }
                tmem_st_frag(tl + sreg + (uint32_t)(t * sh.dcol + c0), sv);
                if (in_b) put_block(x, i0b, c0, true);
              } else if (!last) {
                // T_q = A T_{q-1} / q; S += T_q; operand = T_q, or S after the last term
                float y[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  x[j] = __uint_as_float(dv[j]) * inv;
                  y[j] = __uint_as_float(sv[j]) + x[j];
                  sv[j] = __float_as_uint(y[j]);
                }
                tmem_st_frag(tl + sreg + (uint32_t)(t * sh.dcol + c0), sv);
                if (in_b) put_block(q < sh.order ? x : y, i0b, c0, q < sh.order);
              } else {
                // Phi' = S + (E - I) S
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  const int i = i0b + lane_of(j), c = c0 + col_of(j), b = c < sh.Np ? c : c - sh.Np;
                  if (i < sh.M && b < sh.N) {
                    const float y = __uint_as_float(sv[j]) + __uint_as_float(dv[j]);
                    const int64_t gi = (c < sh.Np ? 0 : plane) + ((int64_t)w * sh.N + b) * sh.M + i;
                    phi_out[gi] = f32_to_f64(y);
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
        if (pre) {
#pragma unroll
          for (int u = 0; u < kXu; ++u)
            if (xo[u] >= 0) xst[xo[u]] = f64_to_f32_rn(xp[u]);
          if (last) mbar_arrive(xfull);   // the next walker's X is staged
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
  s.acol = 2 * s.MT * s.dcol;
  uint32_t need = (uint32_t)(s.acol + (resident ? 4 * 32 * s.KB : 0)), cols = 32;
  s.ecol = (int)need;
  s.eres = resident && need + 2 * 32 * s.KB <= 512u;
  if (s.eres) need += 2 * 32 * s.KB;
  while (cols < need) cols <<= 1;
  s.tcols = cols;
  s.order = c.opt.taylor_order;
  s.Nw = c.Nw;
  s.resident = resident;
  s.ring_off = 0;
  // (the staging covers kXu elements per epilogue thread and round)
  s.xs = resident && s.eres && s.n2 * s.M <= kXu * 32 * 8 * (s.order + 2);
  s.xs_ld = s.M + 4;   // rows 4 floats apart: the fragment reads below fall in distinct banks
  s.ares_off = s.xs ? (s.n2 * s.xs_ld * 4 + 1023) / 1024 * 1024 : nst * kTile;
  s.bhi_off = s.ares_off + (resident ? 4 * s.KB * kTile : 0);
  s.blo_off = s.bhi_off + s.KB * s.bkb;
  s.bar_off = s.blo_off + s.KB * s.bkb;
  s.smem_bytes = s.bar_off + 8 * (2 * kMaxStages + 7) + 16 + 1024;
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
  return s.smem_bytes <= 227 * 1024 && s.tcols <= (two_per_sm(s) ? 256u : 512u);
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
