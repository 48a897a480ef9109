// Latency-oriented FP64 walker kernels for the split-precision step: overlap / LU / weight
// update and modified Gram-Schmidt with the small dense linear algebra (N_s <= 16) in one
// warp, synchronised with __syncwarp only.  Overlaps (FP64, or FP32 pairs when Phi is
// FP32-exact), determinants, ratios, weights and Gram-Schmidt are FP64; Theta = Phi O^{-1}
// is formed in FP32.  Also the fields kernel of the split-precision step.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cuda_bf16.h>

#include "device_util.cuh"
#include "internal.h"

namespace afq {
namespace {

constexpr int kNsMax = 16;   // spin block size handled by the warp LU
constexpr int kPad = 4;      // column padding (elements) of the shared copies of Phi
constexpr int kLd = 24;      // row stride (doubles) of the in-place LU factors of blocks above 8:
                             // the trailing updates' accesses (2 rows per pass) fall in distinct banks

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}

struct FastOvArgs {
  const double* src;  // [2][Nw][N][M]  (propagated walkers in update mode)
  const float* src32; // the same in FP32 (update mode, may be null): no conversions needed,
                      // and the overlap is summed in double-float FP32 arithmetic
  const float* psih;  // psi = psih + psil (FP32 pair, [N][M])
  const float* psil;
  double* phi;
  float* theta32;
  __nv_bfloat16* op_hi;
  __nv_bfloat16* op_lo;
  int Kp;
  const double* psi;  // [N][M]
  double* logO;
  double* w;
  int* alive;
  const double* aux;
  int* flags;
  double* det;        // [Nw][8]: per spin the determinant mantissa (re, im), the summed
                      // power-of-two exponent, the singular flag (k_overlap_fast -> k_overlap_weights)
  int M, N, n_up, Nw, mode, free_proj;
  int fp64_copy;      // 1: Phi also staged in FP64 shared memory (every mode but the FP32 update)
  double log_shift;
};

// (s, c) += (s2, c2) for unevaluated FP32 pairs, the leading sum error-free (two-sum)
__device__ __forceinline__ void df_add(float& s, float& c, float s2, float c2) {
  const float t = __fadd_rn(s, s2);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, c2));
}

// Scalar-type details of the LU: the integer magnitude key of a component (the high word of
// |x|, monotone in |x|) and its bounds (below: zero or subnormal, above: non-finite), the
// biased exponent, the exact power of two 2^(bias - e), and a reciprocal.
template <typename T> struct LuT;
template <> struct LuT<double> {
  static constexpr unsigned kMin = 0x00100000u, kInf = 0x7ff00000u;
  static constexpr int kMaxE = 2046;
  static __device__ __forceinline__ unsigned key(double x) { return (unsigned)__double2hiint(x) & 0x7fffffffu; }
  static __device__ __forceinline__ int expo(double x) { return (__double2hiint(x) >> 20) & 0x7ff; }
  static __device__ __forceinline__ double pow2(int eh) { return __hiloint2double((2046 - eh) << 20, 0); }
  static __device__ __forceinline__ int bias() { return 1023; }
  static __device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }
  static __device__ __forceinline__ double fm(double a, double b, double c) { return fma(a, b, c); }
};
template <> struct LuT<float> {
  static constexpr unsigned kMin = 0x00800000u, kInf = 0x7f800000u;
  static constexpr int kMaxE = 254;
  static __device__ __forceinline__ unsigned key(float x) { return __float_as_uint(x) & 0x7fffffffu; }
  static __device__ __forceinline__ int expo(float x) { return (int)((__float_as_uint(x) >> 23) & 0xffu); }
  static __device__ __forceinline__ float pow2(int eh) { return __uint_as_float((unsigned)(254 - eh) << 23); }
  static __device__ __forceinline__ int bias() { return 127; }
  static __device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
  static __device__ __forceinline__ float fm(float a, float b, float c) { return fmaf(a, b, c); }
};

// LU factorisation with partial (row) pivoting of one spin block, P O = L U, in FP64 (or FP32,
// T = float) by W lanes of a warp (W = 16: both halves of the warp factorise one block each, in step; W = 32:
// one block per warp).  Pivot k interchanges whole rows, scales row k right of the diagonal by
// 1 / pivot (U is unit upper triangular), stores 1 / pivot on the diagonal and updates the
// trailing block; L, with the pivots as its diagonal, is left below the diagonal.  The pivots
// and the determinant are those of Gauss-Jordan elimination with the same pivoting.  Every
// FP64 warp instruction occupies the FP64 pipe whatever its active lanes, so the per-pivot
// scalar work is short and runs in all lanes: the pivot is chosen on an integer magnitude key
// (the high word of |re| or |im|, monotone in the magnitude), the determinant is the product
// of the pivots renormalised by an exact power of two built from its exponent bits, the row
// scale uses one reciprocal, and row blocks of the trailing update that no lane needs are
// skipped.  Each complex update is 4 FP64 fused multiply-adds.  Lane l owns column l % ns and
// rows l / ns + q (W / ns), q < Q.  kmax: the larger block of the warp (uniform loop bound).
template <int W, int Q, int LD, typename T = double>
__device__ __forceinline__ void lu_block(T* __restrict__ ar, T* __restrict__ ai, int l,
                                         int ns, int kmax, int* __restrict__ piv, T& dr,
                                         T& di, int& dexp, bool& bad) {
  using S = LuT<T>;
  const int nsd = ns > 0 ? ns : 1, RS = W / nsd;
  const int c = l % nsd, r0 = l / nsd;
  const bool active = ns > 0 && r0 < RS;
  dr = T(1);
  di = T(0);
  dexp = 0;
  bad = false;
  for (int k = 0; k < kmax; ++k) {
    const bool live = k < ns && !bad;
    unsigned key = 0u;
    if (live && l >= k && l < ns) {
      const unsigned hr = S::key(ar[l * LD + k]);
      const unsigned hi = S::key(ai[l * LD + k]);
      key = hr > hi ? hr : hi;
    }
    int p = l;
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) {
      const unsigned ok = __shfl_xor_sync(0xffffffffu, key, o);
      const int op = __shfl_xor_sync(0xffffffffu, p, o);
      if (ok > key || (ok == key && op < p)) { key = ok; p = op; }
    }
    // zero, subnormal-only or non-finite column: singular for this kernel
    if (live && (key < S::kMin || key >= S::kInf)) bad = true;
    const bool go = live && !bad;
    if (go && l == 0) piv[k] = p;
    if (go && p != k && l < ns) {
      T t = ar[k * LD + l]; ar[k * LD + l] = ar[p * LD + l]; ar[p * LD + l] = t;
      t = ai[k * LD + l]; ai[k * LD + l] = ai[p * LD + l]; ai[p * LD + l] = t;
    }
    __syncwarp();
    const T vr = go ? ar[k * LD + k] : T(1), vi = go ? ai[k * LD + k] : T(0);
    {
      const T tr = S::fm(dr, vr, -di * vi);
      T ti = S::fm(dr, vi, di * vr);
      T trr = tr;
      if (go && p != k) { trr = -tr; ti = -ti; }
      if (go) { dr = trr; di = ti; }
      const int e1 = S::expo(dr), e2 = S::expo(di);
      const int eh = e1 > e2 ? e1 : e2;
      if (eh > 0 && eh < S::kMaxE) {
        const T sc = S::pow2(eh);   // 2^(bias - eh), exact
        dr *= sc;
        di *= sc;
        dexp += eh - S::bias();
      }
    }
    const T rinv = S::rcp(S::fm(vr, vr, vi * vi));
    const T ir = vr * rinv, ii = -vi * rinv;          // 1 / pivot
    __syncwarp();
    if (go && l >= k && l < ns) {
      const T xr = ar[k * LD + l], xi = ai[k * LD + l];
      ar[k * LD + l] = (l == k) ? ir : S::fm(xr, ir, -xi * ii);
      ai[k * LD + l] = (l == k) ? ii : S::fm(xr, ii, xi * ir);
    }
    __syncwarp();
    // A[r][c] -= A[r][k] U[k][c] for r, c > k: column k and row k are not written, so no
    // synchronisation separates these reads from the update
    const bool colk = go && active && c > k;
    const int qf = colk ? max(0, (k + 1 - r0 + RS - 1) / RS) : Q;
    const int q0 = __reduce_min_sync(0xffffffffu, qf);
    const T kr = colk ? ar[k * LD + c] : T(0), ki = colk ? ai[k * LD + c] : T(0);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      if (q >= q0) {
        const int r = r0 + q * RS;
        if (colk && r < ns && r > k) {
          const T fr = ar[r * LD + k], fi = ai[r * LD + k];
          ar[r * LD + c] = S::fm(-fr, kr, S::fm(fi, ki, ar[r * LD + c]));
          ai[r * LD + c] = S::fm(-fr, ki, S::fm(-fi, kr, ai[r * LD + c]));
        }
      }
    }
    __syncwarp();
  }
}

// One CTA (128 or 256 threads) per walker.  Shared: phi [2][N][M + kPad] in FP64 (not in the
// FP32 update), per spin the overlap matrix factorised in place (re and im [NSM][LDA], FP64),
// FP32 copies of phi and of the factors.
// NSM: the larger spin block is at most 8 (both blocks factorised by warp 0, 16 lanes each) or
// 16 (one warp per block, ROWS = ceil(ns / (32 / ns)) rows per lane, 4 or 8).
template <int ROWS, int NSM>
__global__ void __launch_bounds__(256) k_overlap_fast(FastOvArgs a) {
  extern __shared__ double smo[];
  const int wk = blockIdx.x, tid = threadIdx.x, M = a.M, N = a.N, NM = N * M;
  // shared copies of Phi keep each column M + 4 apart: the overlap sums read 8 columns per
  // warp, which then fall in distinct banks
  const int MP = M + kPad, NMP = N * MP;
  // in-place factors of a spin block: NSM rows of LDA doubles per re / im plane; blocks of at
  // most 8 use a stride of 8, which puts the two row sets of a 16-lane half in disjoint banks
  constexpr int LDA = NSM == 8 ? 8 : kLd, PLN = NSM * LDA, SPB = 2 * PLN;
  const int lane = tid & 31, warp = tid >> 5;
  double* pr = smo;            // [N][MP] (only when a.fp64_copy: the FP64 overlap sums)
  double* pi = pr + NMP;       // [N][MP]
  double* aug = a.fp64_copy ? pi + NMP : smo;   // LU factors: spin s at aug + s * SPB, re, im [NSM][LDA]
  // FP32 copies for Theta: converting once here keeps double->float conversions (which run
  // on the FP64 pipe) off the Theta loop
  float* pfr = a.fp64_copy ? reinterpret_cast<float*>(aug + 2 * SPB)   // [N][MP]
                           : reinterpret_cast<float*>(smo);
  float* pfi = pfr + NMP;
  float* invf = pfi + NMP;     // spin s at invf + s * 2 * 16 * 16: re [16][16], im [16][16]
  __shared__ double s_det[2][2];   // per spin: determinant mantissa (re, im) ...
  __shared__ int s_dexp[2];        // ... and its power-of-two exponent
  __shared__ int s_bad[2];
  __shared__ int s_piv[2][kNsMax];
  __shared__ unsigned long long s_perm[2];   // row j of P O_s is row (s_perm >> 4 j) & 15 of O_s
  const bool live = a.alive[wk] != 0;
  // a dead walker keeps its Phi, so its overlap, Theta and operand rows do not change: the
  // update skips it (k_overlap_weights too)
  if (a.mode == OV_UPDATE && !live) return;
  const bool upd = (a.mode == OV_UPDATE) && live;
  const double* src = upd ? a.src : a.phi;
  const int64_t plane = (int64_t)a.Nw * NM, wbase = (int64_t)wk * NM;
  const bool f32 = upd && a.src32 != nullptr;
  const bool inplace = upd && a.src == a.phi;   // the propagator already wrote Phi
  if (f32 && inplace) {
    // the FP32 walker into the padded shared layout by asynchronous copies, all in flight at
    // once (16-byte chunks when the columns allow, else 4-byte words)
    const uint32_t sr0 = smem_addr(pfr), si0 = smem_addr(pfi);
    const float* g0 = a.src32 + wbase;
    if ((M & 3) == 0) {
      const int q = M >> 2;
      for (int c = tid; c < N * q; c += blockDim.x) {
        const int n = c / q, i = (c - n * q) << 2;
        cp_async16(sr0 + 4u * (uint32_t)(n * MP + i), g0 + n * M + i);
        cp_async16(si0 + 4u * (uint32_t)(n * MP + i), g0 + plane + n * M + i);
      }
    } else {
      for (int e = tid; e < NM; e += blockDim.x) {
        const uint32_t es = (uint32_t)(e + (e / M) * kPad);
        cp_async4(sr0 + 4u * es, g0 + e);
        cp_async4(si0 + 4u * es, g0 + plane + e);
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else
  for (int e = tid; e < NM; e += blockDim.x) {
    const int es = e + (e / M) * kPad;   // (n, i) in the padded layout
    if (f32) {
      pfr[es] = a.src32[wbase + e];
      pfi[es] = a.src32[plane + wbase + e];
      if (!inplace) {            // the propagated walker becomes the walker: no dependence on O
        a.phi[wbase + e] = src[wbase + e];
        a.phi[plane + wbase + e] = src[plane + wbase + e];
      }
    } else {
      const double xr = src[wbase + e], xi = src[plane + wbase + e];
      if (upd && !inplace) {
        a.phi[wbase + e] = xr;
        a.phi[plane + wbase + e] = xi;
      }
      pr[es] = xr;               // the FP64 copy feeds the FP64 overlap sums
      pi[es] = xi;
      pfr[es] = (float)xr;
      pfi[es] = (float)xi;
    }
  }
  if (tid < 2) { s_det[tid][0] = 1.0; s_det[tid][1] = 0.0; s_dexp[tid] = 0; s_bad[tid] = 0; }
  __syncthreads();
  // O_s[a][b] = sum_i psi[n0+a][i] phi[n0+b][i]; 4 threads per entry, shuffle-combined
  const int nu = a.n_up, nd = N - nu, nn = nu * nu + nd * nd;
  for (int base = 0; base < nn * 4; base += blockDim.x) {
    const int q = base + tid, ent = q >> 2, part = q & 3;
    double re = 0.0, im = 0.0;
    float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;   // FP32-pair partial sums (update mode)
    int sp = 0, r = 0, c = 0;
    if (ent < nn) {
      if (ent < nu * nu) { r = ent / nu; c = ent % nu; }
      else { sp = 1; const int e2 = ent - nu * nu; r = e2 / nd; c = e2 % nd; }
      const int n0 = sp ? nu : 0;
      if (f32) {
        // phi is FP32 here (the propagator's FP32 output): FP32 products of psi (rounded to
        // FP32) and phi, summed in FP32 (~2^-24 relative to sum |terms| per part; the log
        // determinant then carries ~1e-6 of rounding, far below the step's other FP32 and
        // split-BF16 errors); the FP64 pipe sees only the final conversions
        const float* hs = a.psih + (int64_t)(n0 + r) * M;
        const float* xr = pfr + (n0 + c) * MP;
        const float* xi = pfi + (n0 + c) * MP;
        for (int i = part; i < M; i += 4) {
          const float h = __ldg(hs + i);
          sr = fmaf(h, xr[i], sr);
          si = fmaf(h, xi[i], si);
        }
      } else {
        const double* ps = a.psi + (int64_t)(n0 + r) * M;
        const double* fr = pr + (n0 + c) * MP;
        const double* fi = pi + (n0 + c) * MP;
        for (int i = part; i < M; i += 4) {
          const double p = __ldg(ps + i);
          re = fma(p, fr[i], re);
          im = fma(p, fi[i], im);
        }
      }
    }
    // combine the 4 partial sums of each entry (every lane takes part in the shuffles)
    if (f32) {
      // FP32 pairs with error-free additions: the FP64 pipe sees one conversion per component
#pragma unroll
      for (int o = 1; o <= 2; o <<= 1) {
        const float s2r = __shfl_xor_sync(0xffffffffu, sr, o), c2r = __shfl_xor_sync(0xffffffffu, cr, o);
        const float s2i = __shfl_xor_sync(0xffffffffu, si, o), c2i = __shfl_xor_sync(0xffffffffu, ci, o);
        df_add(sr, cr, s2r, c2r);
        df_add(si, ci, s2i, c2i);
      }
      // every lane of the entry holds the combined pair; part 0 converts the real sum and
      // part 1 the imaginary one, so each lane issues 2 conversions and 1 add
      // (FP32 update: the factorisation below runs in FP32 on these)
      const bool odd = part & 1;
      if (ent < nn && part < 2)
        invf[sp * 2 * kNsMax * kNsMax + (odd ? kNsMax * kNsMax : 0) + r * kNsMax + c] =
            (odd ? si : sr) + (odd ? ci : cr);
    } else {
      re += __shfl_xor_sync(0xffffffffu, re, 1);
      im += __shfl_xor_sync(0xffffffffu, im, 1);
      re += __shfl_xor_sync(0xffffffffu, re, 2);
      im += __shfl_xor_sync(0xffffffffu, im, 2);
      if (ent < nn && part == 0) {
        double* ar = aug + sp * SPB;
        double* ai = ar + PLN;
        ar[r * LDA + c] = re;
        ai[r * LDA + c] = im;
      }
    }
  }
  __syncthreads();
  if (f32) {
    // FP32 update: the factors in FP32 in place (they are what the Theta solves read), the
    // determinant as an FP32 mantissa and a power-of-two exponent; log O then carries FP32
    // rounding, which the next step's ratio cancels
    if (NSM == 8) {
      if (warp == 0) {
        const int h = lane >> 4, l16 = lane & 15, ns = h ? nd : nu;
        float* ar = invf + h * 2 * kNsMax * kNsMax;
        float dr, di;
        int dexp;
        bool bad;
        lu_block<16, 4, kNsMax, float>(ar, ar + kNsMax * kNsMax, l16, ns, nu > nd ? nu : nd, s_piv[h],
                                       dr, di, dexp, bad);
        if (l16 == 0) {
          s_det[h][0] = dr;
          s_det[h][1] = di;
          s_dexp[h] = dexp;
          s_bad[h] = bad ? 1 : 0;
        }
      }
    } else if (warp < 2) {
      const int sp = warp, ns = sp ? nd : nu;
      float* ar = invf + sp * 2 * kNsMax * kNsMax;
      float dr, di;
      int dexp;
      bool bad;
      lu_block<32, ROWS, kNsMax, float>(ar, ar + kNsMax * kNsMax, lane, ns, ns, s_piv[sp], dr, di,
                                        dexp, bad);
      if (lane == 0) {
        s_det[sp][0] = dr;
        s_det[sp][1] = di;
        s_dexp[sp] = dexp;
        s_bad[sp] = bad ? 1 : 0;
      }
    }
  } else if (NSM == 8) {
    if (warp == 0) {   // both spin blocks, 16 lanes each
      const int h = lane >> 4, l16 = lane & 15, ns = h ? nd : nu;
      double* ar = aug + h * SPB;
      double dr, di;
      int dexp;
      bool bad;
      lu_block<16, 4, LDA>(ar, ar + PLN, l16, ns, nu > nd ? nu : nd, s_piv[h], dr, di, dexp, bad);
      if (l16 == 0) {
        s_det[h][0] = dr;
        s_det[h][1] = di;
        s_dexp[h] = dexp;
        s_bad[h] = bad ? 1 : 0;
      }
    }
  } else if (warp < 2) {
    const int sp = warp, ns = sp ? nd : nu;
    double* ar = aug + sp * SPB;
    double dr, di;
    int dexp;
    bool bad;
    lu_block<32, ROWS, LDA>(ar, ar + PLN, lane, ns, ns, s_piv[sp], dr, di, dexp, bad);
    if (lane == 0) {
      s_det[sp][0] = dr;
      s_det[sp][1] = di;
      s_dexp[sp] = dexp;
      s_bad[sp] = bad ? 1 : 0;
    }
  }
  __syncthreads();
  const bool bad = s_bad[0] || s_bad[1];
  if (tid < 2) {   // P from the interchanges, in order, as 4-bit row indices
    const int ns = tid ? nd : nu;
    unsigned long long pw = 0xfedcba9876543210ull;
    if (!bad)
      for (int k = 0; k < ns; ++k) {
        const int p = s_piv[tid][k];
        const unsigned long long a = (pw >> (4 * k)) & 15ull, b = (pw >> (4 * p)) & 15ull;
        pw ^= ((a ^ b) << (4 * k)) | ((a ^ b) << (4 * p));
      }
    s_perm[tid] = pw;
  }
  if (!f32)
  for (int e = tid; e < nn; e += blockDim.x) {   // the factors (and 1/pivot) to FP32, once
    int sp = 0, r, c;
    if (e < nu * nu) { r = e / nu; c = e % nu; }
    else { sp = 1; r = (e - nu * nu) / nd; c = (e - nu * nu) % nd; }
    const double* ar = aug + sp * SPB;
    float* fr = invf + sp * 2 * kNsMax * kNsMax;
    fr[r * kNsMax + c] = (float)ar[r * LDA + c];
    fr[kNsMax * kNsMax + r * kNsMax + c] = (float)ar[PLN + r * LDA + c];
  }
  __syncthreads();
  // Theta_s = Phi_s O_s^{-1} = ((Phi_s U^{-1}) L^{-1}) P, one orbital row i of one spin per
  // thread, in FP32: y U = phi_i (U unit upper), z L = y (L lower, 1/pivot on the diagonal),
  // theta_i[perm[j]] = z_j.  Written as the FP32 copy and the split bf16 force-bias operand.
  auto put = [&](int e, float re, float im) {
    const int64_t gi = wbase + e;
    a.theta32[gi] = re;
    a.theta32[plane + gi] = im;
    const int64_t r0 = (int64_t)wk * a.Kp + e, r1 = (int64_t)(a.Nw + wk) * a.Kp + e;
    const __nv_bfloat16 h0 = __float2bfloat16_rn(re), h1 = __float2bfloat16_rn(im);
    a.op_hi[r0] = h0;
    a.op_lo[r0] = __float2bfloat16_rn(re - __bfloat162float(h0));
    a.op_hi[r1] = h1;
    a.op_lo[r1] = __float2bfloat16_rn(im - __bfloat162float(h1));
  };
  if (bad) {
    for (int e = tid; e < NM; e += blockDim.x) put(e, 0.f, 0.f);
  } else {
    for (int t = tid; t < 2 * M; t += blockDim.x) {
      const int sp = t / M, i = t - sp * M, ns = sp ? nd : nu, n0 = sp ? nu : 0;
      const float* Lr = invf + sp * 2 * kNsMax * kNsMax;
      const float* Li = Lr + kNsMax * kNsMax;
      float yr[NSM], yi[NSM];
#pragma unroll
      for (int j = 0; j < NSM; ++j) {
        yr[j] = j < ns ? pfr[(n0 + j) * MP + i] : 0.f;
        yi[j] = j < ns ? pfi[(n0 + j) * MP + i] : 0.f;
      }
#pragma unroll
      for (int j = 1; j < NSM; ++j)
        if (j < ns) {
#pragma unroll
          for (int k = 0; k < j; ++k) {
            const float ur = Lr[k * kNsMax + j], ui = Li[k * kNsMax + j];
            yr[j] = fmaf(-yr[k], ur, fmaf(yi[k], ui, yr[j]));
            yi[j] = fmaf(-yr[k], ui, fmaf(-yi[k], ur, yi[j]));
          }
        }
#pragma unroll
      for (int j = NSM - 1; j >= 0; --j)
        if (j < ns) {
          float tr = yr[j], ti = yi[j];
#pragma unroll
          for (int k = j + 1; k < NSM; ++k)
            if (k < ns) {
              const float lr = Lr[k * kNsMax + j], li = Li[k * kNsMax + j];
              tr = fmaf(-yr[k], lr, fmaf(yi[k], li, tr));
              ti = fmaf(-yr[k], li, fmaf(-yi[k], lr, ti));
            }
          const float pr_ = Lr[j * kNsMax + j], pi_ = Li[j * kNsMax + j];
          yr[j] = fmaf(tr, pr_, -ti * pi_);
          yi[j] = fmaf(tr, pi_, ti * pr_);
        }
      const unsigned long long pw = s_perm[sp];
#pragma unroll
      for (int j = 0; j < NSM; ++j)
        if (j < ns) put((n0 + (int)((pw >> (4 * j)) & 15ull)) * M + i, yr[j], yi[j]);
    }
  }
  // the per-walker scalar work (a log, an atan2, the weight update) runs in k_overlap_weights,
  // one thread per walker: here it would occupy the FP64 pipe for a whole warp per walker
  if (tid < 6) {
    double v = bad ? 1.0 : 0.0;
    if (tid < 4) v = s_det[tid >> 1][tid & 1];
    else if (tid == 4) v = (double)(s_dexp[0] + s_dexp[1]);
    a.det[8 * (int64_t)wk + tid] = v;
  }
}

// Per walker, after k_overlap_fast: log det O, the overlap ratio and the weight update.
__global__ void __launch_bounds__(32) k_overlap_weights(FastOvArgs a) {
  const int wk = blockIdx.x * blockDim.x + threadIdx.x;
  if (wk >= a.Nw) return;
  const bool upd = (a.mode == OV_UPDATE) && a.alive[wk] != 0;
  if (a.mode == OV_UPDATE && !upd) return;
  const double* dt = a.det + 8 * (int64_t)wk;
  const bool bad = dt[5] != 0.0;
  // log det O = log(d_up d_dn) + (e_up + e_dn) ln 2
  const double d0r = dt[0], d0i = dt[1], d1r = dt[2], d1i = dt[3];
  const double pr_ = fma(d0r, d1r, -d0i * d1i), pi_ = fma(d0r, d1i, d0i * d1r);
  const double ld_re = 0.5 * log(fma(pr_, pr_, pi_ * pi_)) + dt[4] * M_LN2;
  const double ld_im = atan2(pi_, pr_);
  if (bad || !isfinite(ld_re) || !isfinite(ld_im)) {
    atomicAdd(a.flags, 1);
    if (upd || a.mode == OV_REFRESH) {
      a.w[wk] = 0.0;
      a.w[a.Nw + wk] = 0.0;
      a.alive[wk] = 0;
    }
    return;
  }
  if (!upd) {
    a.logO[wk] = ld_re;
    a.logO[a.Nw + wk] = ld_im;
    return;
  }
  const double* x = a.aux + 4 * (int64_t)wk;
  const double lr_re = x[0] + ld_re - a.logO[wk];
  const double lr_im = x[1] + ld_im - a.logO[a.Nw + wk];
  const double li_re = lr_re + x[2] + a.log_shift;
  const double li_im = lr_im + x[3];
  a.logO[wk] = ld_re;
  a.logO[a.Nw + wk] = ld_im;
  if (a.free_proj) {
    const double mag = exp(li_re);
    double sn, cs;
    sincos(li_im, &sn, &cs);
    const cplx nw = cmul({a.w[wk], a.w[a.Nw + wk]}, {mag * cs, mag * sn});
    a.w[wk] = nw.re;
    a.w[a.Nw + wk] = nw.im;
  } else {
    const double nw = a.w[wk] * exp(li_re) * fmax(0.0, cos(lr_im));
    if (nw > 0.0) {
      a.w[wk] = nw;
    } else {
      a.w[wk] = 0.0;
      a.alive[wk] = 0;
    }
    a.w[a.Nw + wk] = 0.0;
  }
}

// Modified Gram-Schmidt, one warp per spin block: columns in order, each projection
// removed one at a time (warp-shuffle inner products), then normalised.  FP64.
__global__ void __launch_bounds__(64) k_mgs_warp(double* __restrict__ phi, const int* __restrict__ alive,
                                                 double* __restrict__ logO, int M, int N, int n_up, int Nw) {
  // one warp per walker (two walkers per CTA): lanes 0-15 orthonormalise the spin-up block,
  // lanes 16-31 the spin-down block, so every FP64 instruction serves both spins; dots reduce
  // over 16 lanes.  Columns in order, each projected on the finished ones (modified
  // Gram-Schmidt), then normalised; all arithmetic FP64.
  extern __shared__ double smg[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wk = blockIdx.x * 2 + warp;
  if (wk >= Nw || !alive[wk]) return;
  const int NM = N * M;
  double* vr = smg + (int64_t)warp * 2 * NM;
  double* vi = vr + NM;
  const int64_t plane = (int64_t)Nw * NM, base = (int64_t)wk * NM;
  for (int e = lane; e < NM; e += 32) {
    vr[e] = phi[base + e];
    vi[e] = phi[plane + base + e];
  }
  __syncwarp();
  const int h = lane >> 4, l16 = lane & 15;
  const int n0 = h ? n_up : 0, ns = h ? N - n_up : n_up, nmax = n_up > N - n_up ? n_up : N - n_up;
  double my_sn = 1.0;   // lane j of each half: squared norm of column j before normalisation
  for (int j = 0; j < nmax; ++j) {
    const bool col = j < ns;
    double* xr = vr + (n0 + (col ? j : 0)) * M;
    double* xi = vi + (n0 + (col ? j : 0)) * M;
    for (int q = 0; q < j; ++q) {
      const double* qr = vr + (n0 + q) * M;
      const double* qi = vi + (n0 + q) * M;
      double s0 = 0, s1 = 0;
      if (col)
        for (int i = l16; i < M; i += 16) {
          s0 += qr[i] * xr[i] + qi[i] * xi[i];
          s1 += qr[i] * xi[i] - qi[i] * xr[i];
        }
      for (int o = 8; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      }
      if (col)
        for (int i = l16; i < M; i += 16) {
          const double u = fma(-s0, qr[i], fma(s1, qi[i], xr[i]));
          const double v = fma(-s0, qi[i], fma(-s1, qr[i], xi[i]));
          xr[i] = u;
          xi[i] = v;
        }
      __syncwarp();
    }
    double sn = 0;
    if (col)
      for (int i = l16; i < M; i += 16) sn += xr[i] * xr[i] + xi[i] * xi[i];
    for (int o = 8; o > 0; o >>= 1) sn += __shfl_xor_sync(0xffffffffu, sn, o);
    if (col && l16 == j) my_sn = sn;
    const double inv = col ? rsqrt(sn) : 0.0;
    if (col)
      for (int i = l16; i < M; i += 16) {
        xr[i] *= inv;
        xi[i] *= inv;
      }
    __syncwarp();
  }
  for (int e = lane; e < NM; e += 32) {
    phi[base + e] = vr[e];
    phi[plane + base + e] = vi[e];
  }
  // Phi -> Phi R^{-1} with R upper triangular, diag(R) = the column norms: log <psi_T|phi>
  // drops by sum_j log R_jj (real), and Theta = Phi (Psi^T Phi)^{-1} is unchanged
  if (logO) {
    double v = l16 < ns ? 0.5 * log(my_sn) : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) logO[wk] -= v;
  }
}

// Register-resident modified Gram-Schmidt for M <= 64 and spin blocks of at most 8 (FP64):
// one warp per walker (two per 64-thread CTA), lanes 0-15 the spin-up block, 16-31 the
// spin-down block; lane l holds rows l + 16 r (r < 4) of every column of its block, so the
// projections and norms read no shared memory (the block with fewer columns carries zero
// columns).  Columns in order, each projected on the finished ones, then normalised; log O
// drops by the log of the norms as in k_mgs_warp.
__global__ void __launch_bounds__(64) k_mgs_reg(double* __restrict__ phi, const int* __restrict__ alive,
                                               double* __restrict__ logO, int M, int N, int n_up, int Nw) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wk = blockIdx.x * 2 + warp;
  if (wk >= Nw || !alive[wk]) return;
  const int h = lane >> 4, l16 = lane & 15;
  const int n0 = h ? n_up : 0, ns = h ? N - n_up : n_up;
  const int64_t NM = (int64_t)N * M, plane = (int64_t)Nw * NM, base = (int64_t)wk * NM;
  double xr[8][4], xi[8][4];
#pragma unroll
  for (int c = 0; c < 8; ++c)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = l16 + 16 * r;
      const bool ok = c < ns && i < M;
      const int64_t g = base + (int64_t)(n0 + (ok ? c : 0)) * M + (ok ? i : 0);
      xr[c][r] = ok ? phi[g] : 0.0;
      xi[c][r] = ok ? phi[plane + g] : 0.0;
    }
  double my_sn = 1.0;   // lane j of each half: squared norm of column j before normalisation
#pragma unroll
  for (int j = 0; j < 8; ++j) {
#pragma unroll
    for (int q = 0; q < j; ++q) {
      double s0 = 0.0, s1 = 0.0;   // <q|x_j>
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        s0 = fma(xr[q][r], xr[j][r], fma(xi[q][r], xi[j][r], s0));
        s1 = fma(xr[q][r], xi[j][r], fma(-xi[q][r], xr[j][r], s1));
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        // x_j -= <q|x_j> q: 4 fused multiply-adds per complex element
        xr[j][r] = fma(-s0, xr[q][r], fma(s1, xi[q][r], xr[j][r]));
        xi[j][r] = fma(-s0, xi[q][r], fma(-s1, xr[q][r], xi[j][r]));
      }
    }
    double sn = 0.0;
#pragma unroll
    for (int r = 0; r < 4; ++r) sn = fma(xr[j][r], xr[j][r], fma(xi[j][r], xi[j][r], sn));
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) sn += __shfl_xor_sync(0xffffffffu, sn, o);
    const bool col = j < ns;
    if (col && l16 == j) my_sn = sn;
    const double inv = col ? rsqrt(sn) : 0.0;   // log O below uses sn itself
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      xr[j][r] *= inv;
      xi[j][r] *= inv;
    }
  }
#pragma unroll
  for (int c = 0; c < 8; ++c)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = l16 + 16 * r;
      if (c < ns && i < M) {
        const int64_t g = base + (int64_t)(n0 + c) * M + i;
        phi[g] = xr[c][r];
        phi[plane + g] = xi[c][r];
      }
    }
  if (logO) {
    double v = l16 < ns ? 0.5 * log(my_sn) : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) logO[wk] -= v;
  }
}

// Orthonormalisation of the split-precision path (Sec. II.D) as a Cholesky QR: per spin block,
// Phi_s = Q R with R upper triangular with a positive diagonal, the factors modified
// Gram-Schmidt produces.  The walker is read as FP32 (the precision the propagator keeps), S =
// Phi_s^H Phi_s is summed in FP32 (four threads per group of entries, each over a quarter of
// the orbitals, combined by shuffles) and factorised S = R^H R in FP32, both spins in one warp
// (16 lanes each, lane l owning column l): S carries the FP32 rounding of its sums already, so
// an FP64 factor would add no accuracy, and on this part each warp-wide FP64 instruction
// (square roots and divisions above all) occupies the FP64 pipe for tens of cycles.  Q =
// Phi_s R^{-1} is formed by forward substitution along every orbital row in FP32 and written
// back exactly as FP64.  log O drops by sum_j log R_jj (FP64 logarithms of the FP32 diagonal),
// the R that Q was formed with, so the stored log O and walker agree up to the FP32 rounding
// of Q (~1e-6 in log O, against which the weights are insensitive).  The walkers are
// orthonormalised every few steps, so S is close to the identity and squaring the condition
// number costs nothing.  One 128-thread CTA per walker; shared memory holds the walker as rows
// of float2 (re, im) with a stride of N + 1, the upper triangle of S factorised in place, R as
// float2 and the reciprocals of its diagonal.
__global__ void __launch_bounds__(128) k_mgs_chol(double* __restrict__ phi, const int* __restrict__ alive,
                                                  double* __restrict__ logO, int M, int N, int n_up,
                                                  int Nw) {
  extern __shared__ __align__(16) unsigned char smc[];
  const int wk = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
  if (!alive[wk]) return;
  const int64_t NM = (int64_t)N * M, plane = (int64_t)Nw * NM, base = (int64_t)wk * NM;
  const int RS = N + 1;                                              // row stride (float2)
  float2* X2 = reinterpret_cast<float2*>(smc);                       // [M][N + 1]
  float* Sre = reinterpret_cast<float*>(X2 + (size_t)M * RS);        // [N][N] (block diagonal)
  float* Sim = Sre + (size_t)N * N;
  float2* R2 = reinterpret_cast<float2*>(Sim + (size_t)N * N);       // [N][N]  R in FP32
  float* Rd = reinterpret_cast<float*>(R2 + (size_t)N * N);          // [N]     1 / R_jj
  __shared__ double s_ld;
  // the walker in FP32 (global layout [2][Nw][N][M], i fastest), loads issued in batches
  for (int64_t e0 = tid; e0 < NM; e0 += 4 * blockDim.x) {
    double xr[4], xi[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t e = e0 + u * blockDim.x;
      xr[u] = e < NM ? phi[base + e] : 0.0;
      xi[u] = e < NM ? phi[plane + base + e] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t e = e0 + u * blockDim.x;
      if (e < NM) {
        const int n = (int)(e / M), i = (int)(e % M);
        X2[(size_t)i * RS + n] = make_float2(f64_to_f32_rn(xr[u]), f64_to_f32_rn(xi[u]));
      }
    }
  }
  __syncthreads();
  // upper triangle of S_s[a][b] = sum_i conj(x_ia) x_ib in FP32; unit (s, a, column group of 4,
  // quarter of the orbitals), groups wholly below the diagonal skipped
  const int nu = n_up, nd = N - n_up;
  const int g0 = (nu + 3) / 4, g1 = (nd + 3) / 4;
  const int items = nu * g0 + nd * g1;
  for (int u0 = 0; u0 < 4 * items; u0 += blockDim.x) {
    const int it = (u0 + tid) >> 2, part = (u0 + tid) & 3;
    float sre[4] = {0.f, 0.f, 0.f, 0.f}, sim[4] = {0.f, 0.f, 0.f, 0.f};
    int ca = 0, o = 0, a = 0, b0 = 0, ns = 0;
    bool live = it < items;
    if (live) {
      const bool dn = it >= nu * g0;
      const int r = dn ? it - nu * g0 : it, gq = dn ? g1 : g0;
      ns = dn ? nd : nu;
      o = dn ? nu : 0;
      a = r / gq;
      b0 = 4 * (r % gq);
      live = b0 + 3 >= a;
      ca = o + a;
    }
    if (live)
      for (int i = part; i < M; i += 4) {
        const float2 x = X2[(size_t)i * RS + ca];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (b0 + k >= ns) break;
          const float2 y = X2[(size_t)i * RS + o + b0 + k];
          // conj(x) y = (xr yr + xi yi) + i (xr yi - xi yr)
          sre[k] = fmaf(x.x, y.x, fmaf(x.y, y.y, sre[k]));
          sim[k] = fmaf(x.x, y.y, fmaf(-x.y, y.x, sim[k]));
        }
      }
    // the four quarters of each unit sit in consecutive lanes
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      sre[k] += __shfl_xor_sync(0xffffffffu, sre[k], 1);
      sim[k] += __shfl_xor_sync(0xffffffffu, sim[k], 1);
      sre[k] += __shfl_xor_sync(0xffffffffu, sre[k], 2);
      sim[k] += __shfl_xor_sync(0xffffffffu, sim[k], 2);
    }
    if (live && part == 0)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int b = b0 + k;
        if (b < ns && b >= a) {
          Sre[(size_t)ca * N + o + b] = sre[k];
          Sim[(size_t)ca * N + o + b] = sim[k];
        }
      }
  }
  __syncthreads();
  // S_s = R^H R (upper triangle in place, FP32), warp 0: lanes 0-15 the spin-up block, 16-31
  // the spin-down block, lane l of a half owning column l
  if (tid < 32) {
    const int h = lane >> 4, l = lane & 15, ns = h ? nd : nu, o = h ? nu : 0;
    const int kmax = nu > nd ? nu : nd;
    for (int k = 0; k < kmax; ++k) {
      const bool act = k < ns;
      const float skk = act ? Sre[(size_t)(o + k) * N + o + k] : 1.0f;
      const float d = sqrtf(skk), inv = 1.0f / d;
      if (act && l > k && l < ns) {
        Sre[(size_t)(o + k) * N + o + l] *= inv;
        Sim[(size_t)(o + k) * N + o + l] *= inv;
      }
      if (act && l == k) {
        Sre[(size_t)(o + k) * N + o + k] = d;
        Sim[(size_t)(o + k) * N + o + k] = 0.0f;
      }
      __syncwarp();
      if (act && l > k && l < ns) {
        const float rr = Sre[(size_t)(o + k) * N + o + l], ri = Sim[(size_t)(o + k) * N + o + l];
        for (int m = k + 1; m <= l; ++m) {   // S_ml -= conj(R_km) R_kl
          const float ar = Sre[(size_t)(o + k) * N + o + m], ai = Sim[(size_t)(o + k) * N + o + m];
          Sre[(size_t)(o + m) * N + o + l] -= fmaf(ar, rr, ai * ri);
          Sim[(size_t)(o + m) * N + o + l] -= fmaf(ar, ri, -ai * rr);
        }
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // R in FP32 (upper triangle, zero below) and the reciprocals of its diagonal; log det R of
  // the FP32 R that forms Q
  for (int e = tid; e < N * N; e += blockDim.x) {
    const int k = e / N, l = e % N;
    const bool same = (k < nu) == (l < nu);
    float2 v = make_float2(0.f, 0.f);
    if (same && l >= k) v = make_float2(Sre[e], Sim[e]);
    R2[e] = v;
    if (k == l) Rd[k] = 1.0f / v.x;
  }
  __syncthreads();
  if (tid < 32) {
    double ld = tid < N ? log((double)R2[(size_t)tid * N + tid].x) : 0.0;
    for (int sh = 16; sh > 0; sh >>= 1) ld += __shfl_xor_sync(0xffffffffu, ld, sh);
    if (lane == 0) s_ld = ld;
  }
  // Q = Phi R^{-1} row by row in FP32: q_j = (x_j - sum_{k<j} q_k R_kj) / R_jj, written over the
  // row (row k < j already holds q_k)
  for (int it = tid; it < 2 * M; it += blockDim.x) {
    const bool dn = it >= M;
    const int i = dn ? it - M : it, ns = dn ? nd : nu, o = dn ? nu : 0;
    float2* row = X2 + (size_t)i * RS + o;
    for (int j = 0; j < ns; ++j) {
      float2 x = row[j];
      for (int k = 0; k < j; ++k) {
        const float2 q = row[k], rv = R2[(size_t)(o + k) * N + o + j];
        x.x = fmaf(-q.x, rv.x, fmaf(q.y, rv.y, x.x));
        x.y = fmaf(-q.x, rv.y, fmaf(-q.y, rv.x, x.y));
      }
      const float inv = Rd[o + j];
      row[j] = make_float2(x.x * inv, x.y * inv);
    }
  }
  __syncthreads();
  for (int64_t e = tid; e < NM; e += blockDim.x) {
    const int n = (int)(e / M), i = (int)(e % M);
    const float2 q = X2[(size_t)i * RS + n];
    phi[base + e] = f32_to_f64(q.x);
    phi[plane + base + e] = f32_to_f64(q.y);
  }
  if (logO && tid == 0) logO[wk] -= s_ld;
}

size_t smem_mgs_chol(const Ctx& c) {
  return sizeof(float2) * (size_t)c.M * (c.N + 1) + 2 * sizeof(float) * (size_t)c.N * c.N +
         sizeof(float2) * (size_t)c.N * c.N + sizeof(float) * (size_t)c.N;
}

size_t smem_fast_overlap(const Ctx& c, bool fp64_copy = true) {
  const size_t nmp = (size_t)c.N * (c.M + kPad);
  const bool small = std::max(c.n_up, c.N - c.n_up) <= 8;   // the NSM = 8 factor layout
  const size_t aug = small ? 2 * 2 * 8 * 8 : 2 * 2 * kNsMax * kLd;
  // the FP32 update factorises in the FP32 factor arrays: no FP64 copy of Phi, no FP64 factors
  return sizeof(double) * (fp64_copy ? 2 * nmp + aug : 0) +
         sizeof(float) * (2 * nmp + 2 * 2 * kNsMax * kNsMax);
}
size_t smem_mgs_warp(const Ctx& c) { return sizeof(double) * 4 * (size_t)c.N * c.M; }   // two walkers

}  // namespace

bool fast_walker_kernels_ok(const Ctx& c) {
  return c.n_up <= kNsMax && c.N - c.n_up <= kNsMax && smem_fast_overlap(c) <= 200 * 1024 &&
         smem_mgs_warp(c) <= 200 * 1024;
}

cudaError_t prepare_fast_walker_kernels(const Ctx& c) {
  static SmemLimits lim;
  const size_t so = smem_fast_overlap(c), sm = smem_mgs_warp(c);
  cudaError_t e = lim.raise(0, so, [&] {
    for (auto* f : {k_overlap_fast<4, 8>, k_overlap_fast<4, 16>, k_overlap_fast<8, 16>}) {
      cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)so);
      if (r != cudaSuccess) return r;
    }
    return cudaSuccess;
  });
  if (e != cudaSuccess) return e;
  e = lim.raise(1, sm, [&] {
    return cudaFuncSetAttribute(k_mgs_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  });
  if (e != cudaSuccess) return e;
  const size_t sc = smem_mgs_chol(c);
  if (sc > 200 * 1024) return cudaSuccess;   // too large: the Gram-Schmidt kernels serve
  return lim.raise(2, sc, [&] {
    return cudaFuncSetAttribute(k_mgs_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc);
  });
}

cudaError_t launch_overlap_fast(const Ctx& c, const double* src, int mode, cudaStream_t s,
                                const float* src32, bool with_weights) {
  FastOvArgs a;
  a.src = src;
  a.src32 = c.psi32h ? src32 : nullptr;
  a.psih = c.psi32h;
  a.psil = c.psi32l; a.phi = c.phi; a.theta32 = c.theta32;
  a.op_hi = c.tc_Theta->hi; a.op_lo = c.tc_Theta->lo; a.Kp = c.tc_Theta->Kp;
  a.psi = c.psi; a.logO = c.logO; a.w = c.w; a.alive = c.alive; a.aux = c.aux; a.flags = c.d_flags;
  a.det = c.ovdet;
  a.M = c.M; a.N = c.N; a.n_up = c.n_up; a.Nw = c.Nw; a.mode = mode;
  a.free_proj = c.opt.mode == AFQMC_FREE;
  a.log_shift = -c.opt.dt * (c.c_mf - c.e_trial);
  a.fp64_copy = !(mode == OV_UPDATE && a.src32 != nullptr);
  auto rows = [](int ns) { return ns > 0 ? (ns + 32 / ns - 1) / (32 / ns) : 0; };
  const int nmax = std::max(c.n_up, c.N - c.n_up);
  const int need = std::max(rows(c.n_up), rows(c.N - c.n_up));
  const size_t sm = smem_fast_overlap(c, a.fp64_copy != 0);
  // the FP32 update (FP32-pair sums, smaller shared footprint) runs more CTAs of 128 threads
  // per SM, so more LU warps overlap; the FP64 sums of the other modes use 256
  const int nt = a.fp64_copy ? 256 : 128;
  if (nmax <= 8) k_overlap_fast<4, 8><<<c.Nw, nt, sm, s>>>(a);
  else if (need <= 4) k_overlap_fast<4, 16><<<c.Nw, nt, sm, s>>>(a);
  else k_overlap_fast<8, 16><<<c.Nw, nt, sm, s>>>(a);
  // one warp per CTA: the FP64 chain of each warp gets an SM's FP64 pipe to itself
  if (with_weights) k_overlap_weights<<<(c.Nw + 31) / 32, 32, 0, s>>>(a);
  return cudaGetLastError();
}

bool mgs_chol_ok(const Ctx& c) {
  return c.n_up <= 16 && c.N - c.n_up <= 16 && smem_mgs_chol(c) <= 200 * 1024;
}

cudaError_t launch_mgs_warp(const Ctx& c, cudaStream_t s, bool update_logO) {
  double* lo = update_logO ? c.logO : nullptr;
  if (c.tune_mgs == 1 && mgs_chol_ok(c)) {
    k_mgs_chol<<<c.Nw, 128, smem_mgs_chol(c), s>>>(c.phi, c.alive, lo, c.M, c.N, c.n_up, c.Nw);
    return cudaGetLastError();
  }
  if (c.M <= 64 && c.n_up <= 8 && c.N - c.n_up <= 8)
    k_mgs_reg<<<(c.Nw + 1) / 2, 64, 0, s>>>(c.phi, c.alive, lo, c.M, c.N, c.n_up, c.Nw);
  else
    k_mgs_warp<<<(c.Nw + 1) / 2, 64, smem_mgs_warp(c), s>>>(c.phi, c.alive, lo, c.M, c.N, c.n_up, c.Nw);
  return cudaGetLastError();
}

}  // namespace afq

namespace afq {
namespace {

// Fields for the split-precision step: the same Philox-4x32-10 bits and Box-Muller
// transform as the FP64 kernel, evaluated in FP32; force bias, shifted fields and the
// V_HS coefficients U = i sqrt(dt) c in FP32, written straight into the split bf16
// operand of the tensor-core V_HS GEMM; the two scalar sums accumulate in FP64.
struct FieldArgsM {
  const float* rhobar;    // [2][Nw][X]  (the FP32 output of the force-bias contraction)
  const float* rho_mf;    // [X]
  const double* fields;   // [Nw][X] or null
  __nv_bfloat16* u_hi;    // [(p, w)][Kp]
  __nv_bfloat16* u_lo;
  int Kp;
  double* aux;            // [Nw][4]
  const unsigned long long* step;
  uint2 key;
  uint32_t k0;
  int X, Nw, free_proj;
  float sqrt_dt, fb_cap;
};

__device__ __forceinline__ void put_split(__nv_bfloat16* hi, __nv_bfloat16* lo, int64_t i, float v) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  hi[i] = h;
  lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
}

__global__ void __launch_bounds__(128) k_fields_mixed(FieldArgsM a) {
  __shared__ float2 red[4][4];   // per warp: the 4 sums as FP32 pairs
  const int wk = blockIdx.x, X = a.X;
  const uint32_t t = (uint32_t)(*a.step);
  const int64_t row = (int64_t)wk * X, plane = (int64_t)a.Nw * X;
  const int64_t o0 = (int64_t)wk * a.Kp, o1 = (int64_t)(a.Nw + wk) * a.Kp;
  // sum c_g rho_g (re, im), x.xbar - xbar^2/2 (re, im): FP32 terms summed as unevaluated FP32
  // pairs (error-free additions), converted to FP64 once per walker, so the thin FP64 pipe only
  // sees the final sums
  float ps[4] = {0.f, 0.f, 0.f, 0.f}, pc[4] = {0.f, 0.f, 0.f, 0.f};
  const int npair = (X + 1) / 2;
  for (int j = threadIdx.x; j < npair; j += blockDim.x) {
    float z[2];
    if (a.fields == nullptr) {
      const uint4 r = philox4x32_10(make_uint4((uint32_t)j, a.k0 + (uint32_t)wk, t, 0u), a.key);
      // the top 24 bits of the 53-bit uniforms (their FP32 roundings up to one unit)
      const float u1 = (float)((r.y >> 8) + 1u) * 0x1p-24f;
      const float u2 = (float)(r.w >> 8) * 0x1p-24f;
      const float rad = sqrtf(-2.0f * logf(u1));
      float sn, cs;
      sincospif(2.0f * u2, &sn, &cs);
      z[0] = rad * cs;
      z[1] = rad * sn;
    }
    float s0 = 0.f, s1 = 0.f, f0 = 0.f, f1 = 0.f;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int g = 2 * j + q;
      if (g >= X) break;
      const float x = a.fields ? (float)a.fields[row + g] : z[q];
      float xb_re = 0.f, xb_im = 0.f;
      const float rm = a.rho_mf[g];
      if (!a.free_proj) {
        xb_re = a.sqrt_dt * a.rhobar[plane + row + g];
        xb_im = -a.sqrt_dt * (a.rhobar[row + g] - rm);
        if (a.fb_cap > 0.f) {
          const float m2 = xb_re * xb_re + xb_im * xb_im;
          if (m2 > a.fb_cap * a.fb_cap) {
            const float sc = a.fb_cap * rsqrtf(m2);
            xb_re *= sc;
            xb_im *= sc;
          }
        }
      }
      const float c_re = x - xb_re, c_im = -xb_im;
      put_split(a.u_hi, a.u_lo, o0 + g, -a.sqrt_dt * c_im);
      put_split(a.u_hi, a.u_lo, o1 + g, a.sqrt_dt * c_re);
      s0 = fmaf(c_re, rm, s0);
      s1 = fmaf(c_im, rm, s1);
      f0 += x * xb_re - 0.5f * (xb_re * xb_re - xb_im * xb_im);
      f1 += x * xb_im - xb_re * xb_im;
    }
    df_add(ps[0], pc[0], s0, 0.f);
    df_add(ps[1], pc[1], s1, 0.f);
    df_add(ps[2], pc[2], f0, 0.f);
    df_add(ps[3], pc[3], f1, 0.f);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    for (int o = 16; o > 0; o >>= 1) {
      const float s2 = __shfl_xor_sync(0xffffffffu, ps[q], o), c2 = __shfl_xor_sync(0xffffffffu, pc[q], o);
      df_add(ps[q], pc[q], s2, c2);
    }
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 4; ++q) red[wid][q] = make_float2(ps[q], pc[q]);
  __syncthreads();
  if (threadIdx.x == 0) {
    // the warps' pairs added as FP32 pairs too; the FP64 pipe sees one add per sum
    double acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float s = red[0][q].x, c = red[0][q].y;
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) df_add(s, c, red[w][q].x, red[w][q].y);
      acc[q] = (double)s + (double)c;
    }
    double* o = a.aux + 4 * (int64_t)wk;
    o[0] = (double)a.sqrt_dt * acc[1];
    o[1] = -(double)a.sqrt_dt * acc[0];
    o[2] = acc[2];
    o[3] = acc[3];
  }
}

}  // namespace

cudaError_t launch_fields_mixed(const Ctx& c, const double* fields, cudaStream_t s) {
  FieldArgsM a;
  a.rhobar = c.rhobar32; a.rho_mf = c.rho_mf32; a.fields = fields;
  a.u_hi = c.tc_U->hi; a.u_lo = c.tc_U->lo; a.Kp = c.tc_U->Kp; a.aux = c.aux; a.step = c.d_step;
  a.key = make_uint2((uint32_t)(c.opt.seed & 0xffffffffull), (uint32_t)(c.opt.seed >> 32));
  a.k0 = (uint32_t)c.opt.walker_offset;
  a.X = c.X; a.Nw = c.Nw; a.free_proj = c.opt.mode == AFQMC_FREE;
  a.sqrt_dt = (float)c.sqrt_dt; a.fb_cap = (float)c.opt.fb_cap;
  k_fields_mixed<<<c.Nw, 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace afq
