// Per-walker kernels of the propagation step.  One CTA owns one walker's
// determinant, so every small dense operation (overlap, Gauss-Jordan inverse,
// Taylor products, Gram-Schmidt, exchange trace) runs out of shared memory with
// coalesced loads from the planar walker layout [2][Nw][N][M].
#include <cmath>
#include <cuda_bf16.h>
#include "device_util.cuh"
#include "internal.h"

namespace afq {

namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------
// Overlap, log-determinant, inverse and Theta (Eqs. 6-7 ingredients), plus the
// phaseless / free-projection weight update of Sec. II.A and II.D.
//   O_s = Psi_s^T Phi_s (Cauchy-Binet overlap per spin), log O = sum_s log det O_s,
//   Theta_s = Phi_s O_s^{-1}.
// mode OV_UPDATE, live walker:  src holds the propagated Phi'; it becomes Phi, and
//   R = s O(Phi')/O(Phi), I = R exp(x.xbar - xbar^2/2) exp(-dt (C - E_T)),
//   phaseless: w <- w |I| max(0, cos arg R) (w <= 0: dead for good); free: w <- w I.
// mode OV_UPDATE, dead walker and OV_REFRESH: Theta and log O recomputed from Phi.
// A singular or non-finite overlap kills the walker (weight 0) and is counted.
// ---------------------------------------------------------------------------
struct OverlapArgs {
  float* theta32;              // split-precision mode: Theta in FP32 [2][Nw][N][M]
  __nv_bfloat16* op_hi;        // split-precision mode: force-bias operand rows [(p,w)][Kp]
  __nv_bfloat16* op_lo;
  int Kp;
  const double* src;   // [2][Nw][N][M]
  double* phi;         // [2][Nw][N][M]
  double* theta;       // [2][Nw][N][M]
  const double* psi;   // [N][M]
  double* logO;        // [2][Nw]
  double* w;           // [2][Nw]
  int* alive;          // [Nw]
  const double* aux;   // [Nw][4]
  int* flags;
  int M, N, n_up, Nw, mode, free_proj;
  double log_shift;    // -dt (C - E_T)
  // mode OV_DET (determinants of a multi-determinant trial, grid row blockIdx.y = d): psi,
  // theta and logO of determinant d start d * det_* elements on; 0 for a single determinant
  int64_t det_psi, det_theta, det_logO;
};

// MIXED: Theta = Phi O^{-1} is formed in FP32 (O, its inverse and log det stay FP64) and
// written as FP32 plus the split bf16 operand of the force-bias tensor-core GEMM.
template <bool MIXED>
__global__ void __launch_bounds__(kThreads) k_overlap(OverlapArgs a) {
  extern __shared__ double sm[];
  const int wk = blockIdx.x, tid = threadIdx.x, M = a.M, N = a.N;
  const int nmax = max(a.n_up, N - a.n_up);
  double* ph = sm;                       // [2][nmax][M]
  double* aug = ph + 2 * nmax * M;       // [2][nmax][2*nmax]   [O | I] -> [I | O^-1]
  double* fac = aug + 4 * nmax * nmax;   // [2 + 2*nmax]: pivot inverse, then column k
  __shared__ double s_ld[2];
  __shared__ int s_piv, s_bad;

  const bool live = a.alive[wk] != 0;
  // OV_DET: overlap, log det and Theta of determinant blockIdx.y only (no weight update)
  const double* psi_d = a.psi + blockIdx.y * a.det_psi;
  double* theta_d = a.theta + blockIdx.y * a.det_theta;
  double* logO_d = a.logO + blockIdx.y * a.det_logO;
  const bool upd = (a.mode == OV_UPDATE) && live;
  const double* src = (upd || (a.mode == OV_DET && a.src)) ? a.src : a.phi;
  const int64_t plane = (int64_t)a.Nw * N * M;
  const int64_t wbase = (int64_t)wk * N * M;
  if (tid == 0) { s_ld[0] = 0.0; s_ld[1] = 0.0; s_bad = 0; }

  for (int sp = 0; sp < 2; ++sp) {
    const int n0 = sp == 0 ? 0 : a.n_up, ns = sp == 0 ? a.n_up : N - a.n_up;
    if (ns == 0) continue;
    const int w2 = 2 * ns;
    __syncthreads();
    for (int e = tid; e < ns * M; e += blockDim.x) {
      const int64_t gi = wbase + (int64_t)n0 * M + e;
      ph[e] = src[gi];
      ph[nmax * M + e] = src[plane + gi];
    }
    __syncthreads();
    // [O | I]
    for (int e = tid; e < ns * w2; e += blockDim.x) {
      const int r = e / w2, c = e % w2;
      double re = 0, im = 0;
      if (c < ns) {
        const double* pr = psi_d + (int64_t)(n0 + r) * M;
        const double* fr = ph + c * M;
        const double* fi = ph + nmax * M + c * M;
        for (int i = 0; i < M; ++i) {
          const double p = __ldg(pr + i);
          re = fma(p, fr[i], re);
          im = fma(p, fi[i], im);
        }
      } else {
        re = (c - ns == r) ? 1.0 : 0.0;
      }
      aug[r * w2 + c] = re;
      aug[ns * w2 + r * w2 + c] = im;
    }
    __syncthreads();
    double* ar = aug;
    double* ai = aug + ns * w2;
    // Gauss-Jordan with partial pivoting
    for (int k = 0; k < ns; ++k) {
      if (tid == 0) {
        int p = k;
        double best = -1.0;
        for (int r = k; r < ns; ++r) {
          const double m2 = ar[r * w2 + k] * ar[r * w2 + k] + ai[r * w2 + k] * ai[r * w2 + k];
          if (m2 > best) { best = m2; p = r; }
        }
        if (!(best > 0.0) || !isfinite(best)) s_bad = 1;
        s_piv = p;
      }
      __syncthreads();
      if (s_bad) break;
      const int p = s_piv;
      if (p != k)
        for (int c = tid; c < w2; c += blockDim.x) {
          double t = ar[k * w2 + c]; ar[k * w2 + c] = ar[p * w2 + c]; ar[p * w2 + c] = t;
          t = ai[k * w2 + c]; ai[k * w2 + c] = ai[p * w2 + c]; ai[p * w2 + c] = t;
        }
      __syncthreads();
      if (tid == 0) {
        const double pr = ar[k * w2 + k], pi = ai[k * w2 + k];
        s_ld[0] += 0.5 * log(pr * pr + pi * pi);
        s_ld[1] += atan2(pi, pr) + (p != k ? M_PI : 0.0);
        const cplx inv = cinv({pr, pi});
        fac[0] = inv.re;
        fac[1] = inv.im;
      }
      __syncthreads();
      const cplx inv = {fac[0], fac[1]};
      for (int c = tid; c < w2; c += blockDim.x) {
        const cplx v = cmul({ar[k * w2 + c], ai[k * w2 + c]}, inv);
        ar[k * w2 + c] = v.re;
        ai[k * w2 + c] = v.im;
      }
      __syncthreads();
      for (int r = tid; r < ns; r += blockDim.x) {
        fac[2 + 2 * r] = ar[r * w2 + k];
        fac[3 + 2 * r] = ai[r * w2 + k];
      }
      __syncthreads();
      for (int e = tid; e < ns * w2; e += blockDim.x) {
        const int r = e / w2, c = e % w2;
        if (r == k) continue;
        const cplx f = {fac[2 + 2 * r], fac[3 + 2 * r]};
        const cplx v = cmul(f, {ar[k * w2 + c], ai[k * w2 + c]});
        ar[e] -= v.re;
        ai[e] -= v.im;
      }
      __syncthreads();
    }
    __syncthreads();
    const bool bad = s_bad != 0;
    // Theta_s[:, b] = sum_c Phi_s[:, c] Oinv[c][b]; copy Phi' into Phi for live updates
    for (int e = tid; e < ns * M; e += blockDim.x) {
      const int b = e / M, i = e % M;
      const int64_t gi = wbase + (int64_t)(n0 + b) * M + i;
      if (MIXED) {
        float re = 0.f, im = 0.f;
        if (!bad)
          for (int c = 0; c < ns; ++c) {
            const float xr = (float)ph[c * M + i], xi = (float)ph[nmax * M + c * M + i];
            const float orr = (float)ar[c * w2 + ns + b], oi = (float)ai[c * w2 + ns + b];
            re = fmaf(xr, orr, fmaf(-xi, oi, re));
            im = fmaf(xr, oi, fmaf(xi, orr, im));
          }
        a.theta32[gi] = re;
        a.theta32[plane + gi] = im;
        const int64_t col = (int64_t)(n0 + b) * M + i;
        const int64_t r0 = (int64_t)wk * a.Kp + col, r1 = (int64_t)(a.Nw + wk) * a.Kp + col;
        const __nv_bfloat16 h0 = __float2bfloat16_rn(re), h1 = __float2bfloat16_rn(im);
        a.op_hi[r0] = h0;
        a.op_lo[r0] = __float2bfloat16_rn(re - __bfloat162float(h0));
        a.op_hi[r1] = h1;
        a.op_lo[r1] = __float2bfloat16_rn(im - __bfloat162float(h1));
      } else {
        double re = 0, im = 0;
        if (!bad)
          for (int c = 0; c < ns; ++c) {
            const double xr = ph[c * M + i], xi = ph[nmax * M + c * M + i];
            const double orr = ar[c * w2 + ns + b], oi = ai[c * w2 + ns + b];
            re = fma(xr, orr, fma(-xi, oi, re));
            im = fma(xr, oi, fma(xi, orr, im));
          }
        theta_d[gi] = re;
        theta_d[plane + gi] = im;
      }
      if (upd) {
        a.phi[gi] = ph[b * M + i];
        a.phi[plane + gi] = ph[nmax * M + b * M + i];
      }
    }
  }
  __syncthreads();
  if (tid != 0) return;
  const bool bad = s_bad != 0;
  const double ld_re = s_ld[0], ld_im = s_ld[1];
  if (bad || !isfinite(ld_re) || !isfinite(ld_im)) {
    if (a.mode == OV_DET) {            // this determinant contributes nothing to the trial
      logO_d[wk] = -INFINITY;
      logO_d[a.Nw + wk] = 0.0;
      return;
    }
    atomicAdd(a.flags, 1);
    if (upd || a.mode == OV_REFRESH) {
      a.w[wk] = 0.0;
      a.w[a.Nw + wk] = 0.0;
      a.alive[wk] = 0;
    }
    return;
  }
  if (!upd) {
    logO_d[wk] = ld_re;
    logO_d[a.Nw + wk] = ld_im;
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
    const cplx f = {mag * cs, mag * sn};
    const cplx nw = cmul({a.w[wk], a.w[a.Nw + wk]}, f);
    a.w[wk] = nw.re;
    a.w[a.Nw + wk] = nw.im;
  } else {
    const double cut = fmax(0.0, cos(lr_im));
    const double nw = a.w[wk] * exp(li_re) * cut;
    if (nw > 0.0) {
      a.w[wk] = nw;
    } else {
      a.w[wk] = 0.0;
      a.alive[wk] = 0;
    }
    a.w[a.Nw + wk] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// Shared auxiliary fields and force bias (Eqs. 4, 8-9; Sec. II.B).  Per walker k:
//   x_g from Philox(key = seed, counter = (g/2, k, t, 0)) or an explicit buffer,
//   xbar_g = -i sqrt(dt) (rhobar_g - <rho_g>_T) capped at |xbar_g| <= fb_cap
//   (phaseless only), c_g = x_g - xbar_g,
//   U_g = i sqrt(dt) c_g  (so that A = sum_g U_g L_g),
//   aux = ( log s = -i sqrt(dt) sum_g c_g <rho_g>_T ,  x.xbar - xbar.xbar/2 ).
// ---------------------------------------------------------------------------
struct FieldArgs {
  const double* rhobar;   // [2][Nw][X]
  const double* rho_mf;   // [X]
  const double* fields;   // [Nw][X] or null
  double* U;              // [2][Nw][X]
  double* aux;            // [Nw][4]
  const unsigned long long* step;
  uint2 key;
  uint32_t k0;            // global pair index of walker 0
  int X, Nw, free_proj;
  double sqrt_dt, fb_cap;
};

__global__ void __launch_bounds__(128) k_fields(FieldArgs a) {
  __shared__ double red[4 * 4 + 4];
  const int wk = blockIdx.x, X = a.X;
  const uint32_t t = (uint32_t)(*a.step);
  const int64_t row = (int64_t)wk * X;
  const int64_t plane = (int64_t)a.Nw * X;
  double acc[4] = {0, 0, 0, 0};   // sum c_g rho_g (re, im), fb (re, im)
  const int npair = (X + 1) / 2;
  for (int j = threadIdx.x; j < npair; j += blockDim.x) {
    double z[2];
    if (a.fields == nullptr) {
      const uint4 r = philox4x32_10(make_uint4((uint32_t)j, a.k0 + (uint32_t)wk, t, 0u), a.key);
      philox_normal2(r, z[0], z[1]);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int g = 2 * j + q;
      if (g >= X) break;
      const double x = a.fields ? a.fields[row + g] : z[q];
      double xb_re = 0.0, xb_im = 0.0;
      if (!a.free_proj) {
        xb_re = a.sqrt_dt * a.rhobar[plane + row + g];
        xb_im = -a.sqrt_dt * (a.rhobar[row + g] - a.rho_mf[g]);
        if (a.fb_cap > 0.0) {
          const double m2 = xb_re * xb_re + xb_im * xb_im;
          if (m2 > a.fb_cap * a.fb_cap) {
            const double sc = a.fb_cap / sqrt(m2);
            xb_re *= sc;
            xb_im *= sc;
          }
        }
      }
      const double c_re = x - xb_re, c_im = -xb_im;
      a.U[row + g] = -a.sqrt_dt * c_im;
      a.U[plane + row + g] = a.sqrt_dt * c_re;
      const double rm = a.rho_mf[g];
      acc[0] = fma(c_re, rm, acc[0]);
      acc[1] = fma(c_im, rm, acc[1]);
      // x xbar - xbar^2 / 2  (unconjugated square)
      acc[2] += x * xb_re - 0.5 * (xb_re * xb_re - xb_im * xb_im);
      acc[3] += x * xb_im - xb_re * xb_im;
    }
  }
  block_sum<4>(acc, red);
  if (threadIdx.x == 0) {
    double* o = a.aux + 4 * (int64_t)wk;
    // log s = -i sqrt(dt) (S_re + i S_im) = sqrt(dt) S_im - i sqrt(dt) S_re
    o[0] = a.sqrt_dt * acc[1];
    o[1] = -a.sqrt_dt * acc[0];
    o[2] = acc[2];
    o[3] = acc[3];
  }
}

// ---------------------------------------------------------------------------
// Taylor exponential (the middle factor of Eq. 11 as a truncated series):
//   Phi <- sum_{m=0}^{n} A^m Phi / m!  by repeated products, A complex symmetric,
//   read from its packed upper triangle.  Terms live in shared memory ([row][col],
//   column fastest, so a warp's reads of one term row are conflict-free); the
//   running sum lives in registers, at most OPT outputs per thread.
// ---------------------------------------------------------------------------
template <int OPT>
__global__ void __launch_bounds__(kThreads) k_taylor(double* __restrict__ phi, const double* __restrict__ Ap,
                                                     int M, int N, int Nw, int64_t P, int order) {
  extern __shared__ double sm[];
  const int wk = blockIdx.x, tid = threadIdx.x, NM = N * M;
  double* tr = sm;             // [M][N]  current term (re)
  double* ti = tr + NM;        // [M][N]  current term (im)
  double* nr = ti + NM;        // next term
  double* ni = nr + NM;
  const int64_t plane = (int64_t)Nw * NM;
  const int64_t base = (int64_t)wk * NM;
  const double* ar = Ap + (int64_t)wk * P;
  const double* ai = Ap + (int64_t)Nw * P + (int64_t)wk * P;
  double acc_r[OPT], acc_i[OPT];
#pragma unroll
  for (int q = 0; q < OPT; ++q) {
    const int o = tid + q * kThreads;
    acc_r[q] = acc_i[q] = 0.0;
    if (o < NM) {
      const int i = o / N, b = o % N;
      const int64_t gi = base + (int64_t)b * M + i;
      acc_r[q] = phi[gi];
      acc_i[q] = phi[plane + gi];
      tr[o] = acc_r[q];
      ti[o] = acc_i[q];
    }
  }
  __syncthreads();
  for (int m = 1; m <= order; ++m) {
    const double inv = 1.0 / (double)m;
#pragma unroll
    for (int q = 0; q < OPT; ++q) {
      const int o = tid + q * kThreads;
      if (o < NM) {
        const int i = o / N, b = o % N;
        double sr = 0, si = 0;
        // j < i: A[i][j] = A[j][i] at packed index rb_j + i,  rb_j = j (M-1) - j (j-1)/2
        int64_t rbj = 0;
        for (int j = 0; j < i; ++j) {
          const double xr = __ldg(ar + rbj + i), xi = __ldg(ai + rbj + i);
          const double yr = tr[j * N + b], yi = ti[j * N + b];
          sr = fma(xr, yr, fma(-xi, yi, sr));
          si = fma(xr, yi, fma(xi, yr, si));
          rbj += (M - 1) - j;
        }
        // j >= i: contiguous run of row i
        const int64_t rbi = (int64_t)i * (M - 1) - (int64_t)i * (i - 1) / 2;
        for (int j = i; j < M; ++j) {
          const double xr = __ldg(ar + rbi + j), xi = __ldg(ai + rbi + j);
          const double yr = tr[j * N + b], yi = ti[j * N + b];
          sr = fma(xr, yr, fma(-xi, yi, sr));
          si = fma(xr, yi, fma(xi, yr, si));
        }
        sr *= inv;
        si *= inv;
        nr[o] = sr;
        ni[o] = si;
        acc_r[q] += sr;
        acc_i[q] += si;
      }
    }
    __syncthreads();
    double* t0 = tr; tr = nr; nr = t0;
    double* t1 = ti; ti = ni; ni = t1;
  }
#pragma unroll
  for (int q = 0; q < OPT; ++q) {
    const int o = tid + q * kThreads;
    if (o < NM) {
      const int i = o / N, b = o % N;
      const int64_t gi = base + (int64_t)b * M + i;
      phi[gi] = acc_r[q];
      phi[plane + gi] = acc_i[q];
    }
  }
}

// ---------------------------------------------------------------------------
// Modified Gram-Schmidt per spin block (Sec. II.D): for each column j in order,
// subtract its projections on the already orthonormal columns one at a time,
// then normalise.  Live walkers only; the weight is unchanged.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_mgs(double* __restrict__ phi, const int* __restrict__ alive,
                                             int M, int N, int n_up, int Nw) {
  extern __shared__ double sm[];
  const int wk = blockIdx.x, tid = threadIdx.x;
  if (!alive[wk]) return;
  const int NM = N * M;
  double* vr = sm;
  double* vi = sm + NM;
  double* red = vi + NM;
  const int64_t plane = (int64_t)Nw * NM, base = (int64_t)wk * NM;
  for (int e = tid; e < NM; e += blockDim.x) {
    vr[e] = phi[base + e];
    vi[e] = phi[plane + base + e];
  }
  __syncthreads();
  for (int sp = 0; sp < 2; ++sp) {
    const int n0 = sp == 0 ? 0 : n_up, n1 = sp == 0 ? n_up : N;
    for (int j = n0; j < n1; ++j) {
      double* xr = vr + j * M;
      double* xi = vi + j * M;
      for (int q = n0; q < j; ++q) {
        const double* qr = vr + q * M;
        const double* qi = vi + q * M;
        double s[2] = {0, 0};   // <q|v> = sum conj(q) v
        for (int i = tid; i < M; i += blockDim.x) {
          s[0] += qr[i] * xr[i] + qi[i] * xi[i];
          s[1] += qr[i] * xi[i] - qi[i] * xr[i];
        }
        block_allsum<2>(s, red);
        for (int i = tid; i < M; i += blockDim.x) {
          const double a = xr[i] - (s[0] * qr[i] - s[1] * qi[i]);
          const double b = xi[i] - (s[0] * qi[i] + s[1] * qr[i]);
          xr[i] = a;
          xi[i] = b;
        }
        __syncthreads();
      }
      double s[1] = {0};
      for (int i = tid; i < M; i += blockDim.x) s[0] += xr[i] * xr[i] + xi[i] * xi[i];
      block_allsum<1>(s, red);
      const double inv = 1.0 / sqrt(s[0]);
      for (int i = tid; i < M; i += blockDim.x) {
        xr[i] *= inv;
        xi[i] *= inv;
      }
      __syncthreads();
    }
  }
  for (int e = tid; e < NM; e += blockDim.x) {
    phi[base + e] = vr[e];
    phi[plane + base + e] = vi[e];
  }
}

// ---------------------------------------------------------------------------
// Local energy (Eq. 7 with Wick's theorem), through the half-rotated tensors:
//   E_L = sum_(n,i) htil[n][i] Theta[n][i]
//       + 1/2 sum_g [ (sum_s tr T^s_g)^2 - sum_s sum_ab T^s_g[a][b] T^s_g[b][a] ],
//   T^s_g[a][b] = sum_i Ltil[g][n0+a][i] Theta[n0+b][i]   (= Psi_s^T L_g Theta_s).
// Theta is staged transposed ([i][n]) so a warp reading one row is conflict-free;
// T for a chunk of G_CH Cholesky vectors is formed in shared memory and reduced
// immediately, never written out.
// ---------------------------------------------------------------------------
constexpr int G_CH = 4;

__global__ void __launch_bounds__(kThreads) k_energy(const double* __restrict__ theta, const double* __restrict__ Ltil,
                                                     const double* __restrict__ htil, double* __restrict__ eloc,
                                                     int M, int N, int n_up, int X, int Nw) {
  extern __shared__ double sm[];
  const int wk = blockIdx.x, tid = threadIdx.x, NM = N * M;
  const int nu = n_up, nd = N - n_up, nn = nu * nu + nd * nd;
  double* thr = sm;                  // [M][N]
  double* thi = thr + NM;            // [M][N]
  double* Tr = thi + NM;             // [G_CH][nn]
  double* Ti = Tr + G_CH * nn;
  double* red = Ti + G_CH * nn;      // 64
  const int64_t plane = (int64_t)Nw * NM, base = (int64_t)wk * NM;
  double acc[4] = {0, 0, 0, 0};      // E1 + 1/2 coul (re, im),  -1/2 exch (re, im)
  for (int e = tid; e < NM; e += blockDim.x) {
    const int n = e / M, i = e % M;
    const double vr = theta[base + e], vi = theta[plane + base + e];
    thr[i * N + n] = vr;
    thi[i * N + n] = vi;
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
      const double* lrow = Ltil + ((int64_t)(g0 + gl) * N + n0 + a) * M;
      double sr = 0, si = 0;
      for (int i = 0; i < M; ++i) {
        const double l = __ldg(lrow + i);
        sr = fma(l, thr[i * N + n0 + b], sr);
        si = fma(l, thi[i * N + n0 + b], si);
      }
      Tr[e] = sr;
      Ti[e] = si;
    }
    __syncthreads();
    for (int e = tid; e < gc * nn; e += blockDim.x) {
      const int gl = e / nn, r = e % nn;
      int et;
      if (r < nu * nu) { const int a = r / nu, b = r % nu; et = b * nu + a; }
      else { const int r2 = r - nu * nu; const int a = r2 / nd, b = r2 % nd; et = nu * nu + b * nd + a; }
      const cplx p = cmul({Tr[e], Ti[e]}, {Tr[gl * nn + et], Ti[gl * nn + et]});
      acc[2] -= 0.5 * p.re;
      acc[3] -= 0.5 * p.im;
    }
    for (int gl = tid; gl < gc; gl += blockDim.x) {
      double cr = 0, ci = 0;
      for (int a = 0; a < nu; ++a) { cr += Tr[gl * nn + a * nu + a]; ci += Ti[gl * nn + a * nu + a]; }
      for (int a = 0; a < nd; ++a) {
        cr += Tr[gl * nn + nu * nu + a * nd + a];
        ci += Ti[gl * nn + nu * nu + a * nd + a];
      }
      acc[0] += 0.5 * (cr * cr - ci * ci);
      acc[1] += cr * ci;
    }
    __syncthreads();
  }
  block_sum<4>(acc, red);
  if (tid == 0) {
    eloc[wk] = acc[0] + acc[2];
    eloc[Nw + wk] = acc[1] + acc[3];
  }
}

// Per-repeat sums for the mixed estimate (Eq. 6): sum_k w_k E_L,k and sum_k w_k over the
// walkers k with floor(k R / Nw) == r.  Phaseless: real weights and Re E_L (Eq. 10).  A dead
// walker (w = 0) adds nothing; it is skipped rather than multiplied by 0, so that the
// non-finite local energy of a walker killed for a non-finite overlap cannot reach the sum.
__global__ void __launch_bounds__(256) k_mixed_sum(const double* __restrict__ w, const double* __restrict__ eloc,
                                                   double* out, const int* slot, int slot_stride,
                                                   int Nw, int R, int free_proj) {
  __shared__ double red[4 * 8 + 4];
  const int r = blockIdx.x;
  const int64_t k0 = ((int64_t)r * Nw + R - 1) / R, k1 = ((int64_t)(r + 1) * Nw + R - 1) / R;
  double acc[4] = {0, 0, 0, 0};
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const double wr = w[k], wi = free_proj ? w[Nw + k] : 0.0;
    if (wr == 0.0 && wi == 0.0) continue;
    const double er = eloc[k], ei = free_proj ? eloc[Nw + k] : 0.0;
    acc[0] += wr * er - wi * ei;
    acc[1] += wr * ei + wi * er;
    acc[2] += wr;
    acc[3] += wi;
  }
  block_sum<4>(acc, red);
  if (threadIdx.x == 0) {
    double* o = out + (slot ? (int64_t)(*slot) * slot_stride : 0) + 4 * r;
    for (int q = 0; q < 4; ++q) o[q] = acc[q];
  }
}

__global__ void k_step_advance(unsigned long long* step, int* meas, int bump_meas) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    if (step) *step += 1ull;
    if (meas && bump_meas) *meas += 1;
  }
}

int opt_for(int NM) { return (NM + kThreads - 1) / kThreads; }

size_t smem_overlap(const Ctx& c) {
  const size_t nmax = c.n_up > c.N - c.n_up ? c.n_up : c.N - c.n_up;
  return sizeof(double) * (2 * nmax * c.M + 4 * nmax * nmax + 2 * nmax + 2);
}
size_t smem_taylor(const Ctx& c) { return sizeof(double) * 4 * (size_t)c.N * c.M; }
size_t smem_mgs(const Ctx& c) { return sizeof(double) * (2 * (size_t)c.N * c.M + 64); }
size_t smem_energy(const Ctx& c) {
  const size_t nu = c.n_up, nd = c.N - c.n_up, nn = nu * nu + nd * nd;
  return sizeof(double) * (2 * (size_t)c.N * c.M + 2 * (size_t)G_CH * nn + 64);
}

// Raise a kernel's dynamic shared-memory limit on the current device to `bytes` if it is
// below; `slot` names the kernel in the record of limits already set.
SmemLimits g_fp64_limits;
template <class F>
cudaError_t ensure_smem(F* f, int slot, size_t bytes) {
  return g_fp64_limits.raise(slot, bytes, [&] {
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  });
}

}  // namespace

// Called once per handle at setup, before any launch or graph capture.
cudaError_t prepare_kernels(const Ctx& c) {
  cudaError_t e;
  if ((e = ensure_smem(k_overlap<false>, 0, smem_overlap(c))) != cudaSuccess) return e;
  if ((e = ensure_smem(k_overlap<true>, 7, smem_overlap(c))) != cudaSuccess) return e;
  if ((e = ensure_smem(k_mgs, 1, smem_mgs(c))) != cudaSuccess) return e;
  if ((e = ensure_smem(k_energy, 2, smem_energy(c))) != cudaSuccess) return e;
  const size_t st = smem_taylor(c);
  if ((e = ensure_smem(k_taylor<2>, 3, st)) != cudaSuccess) return e;
  if ((e = ensure_smem(k_taylor<4>, 4, st)) != cudaSuccess) return e;
  if ((e = ensure_smem(k_taylor<8>, 5, st)) != cudaSuccess) return e;
  if ((e = ensure_smem(k_taylor<16>, 6, st)) != cudaSuccess) return e;
  return cudaSuccess;
}

cudaError_t launch_overlap(const Ctx& c, const double* src, int mode, cudaStream_t s,
                           int n_walkers) {
  OverlapArgs a;
  a.theta32 = c.theta32;
  a.op_hi = c.tc_Theta ? c.tc_Theta->hi : nullptr;
  a.op_lo = c.tc_Theta ? c.tc_Theta->lo : nullptr;
  a.Kp = c.tc_Theta ? c.tc_Theta->Kp : 0;
  a.src = src; a.phi = c.phi; a.theta = c.theta; a.psi = c.psi; a.logO = c.logO; a.w = c.w;
  a.alive = c.alive; a.aux = c.aux; a.flags = c.d_flags;
  a.M = c.M; a.N = c.N; a.n_up = c.n_up; a.Nw = c.Nw; a.mode = mode;
  a.free_proj = c.opt.mode == AFQMC_FREE;
  a.log_shift = -c.opt.dt * (c.c_mf - c.e_trial);
  a.det_psi = a.det_theta = a.det_logO = 0;
  const size_t smem = smem_overlap(c);
  const int grid = n_walkers > 0 ? n_walkers : c.Nw;
  if (c.theta32 && c.tc_Theta) k_overlap<true><<<grid, kThreads, smem, s>>>(a);
  else k_overlap<false><<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_overlap_dets(const Ctx& c, const double* src, cudaStream_t s) {
  if (c.n_det < 1 || c.n_det > 65535) return cudaErrorInvalidValue;
  OverlapArgs a = {};
  a.src = src; a.phi = c.phi; a.alive = c.alive; a.aux = c.aux; a.flags = c.d_flags;
  a.psi = c.md_psi; a.theta = c.md_theta; a.logO = c.md_logO; a.w = c.w;
  a.M = c.M; a.N = c.N; a.n_up = c.n_up; a.Nw = c.Nw; a.mode = OV_DET;
  a.det_psi = (int64_t)c.N * c.M;
  a.det_theta = 2 * (int64_t)c.Nw * c.N * c.M;
  a.det_logO = 2 * (int64_t)c.Nw;
  k_overlap<false><<<dim3(c.Nw, c.n_det), kThreads, smem_overlap(c), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fields(const Ctx& c, const double* fields, cudaStream_t s) {
  FieldArgs a;
  a.rhobar = c.rhobar; a.rho_mf = c.rho_mf; a.fields = fields; a.U = c.U; a.aux = c.aux;
  a.step = c.d_step;
  a.key = make_uint2((uint32_t)(c.opt.seed & 0xffffffffull), (uint32_t)(c.opt.seed >> 32));
  a.k0 = (uint32_t)c.opt.walker_offset;
  a.X = c.X; a.Nw = c.Nw; a.free_proj = c.opt.mode == AFQMC_FREE;
  a.sqrt_dt = c.sqrt_dt; a.fb_cap = c.opt.fb_cap;
  k_fields<<<c.Nw, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_taylor(const Ctx& c, double* phi_io, cudaStream_t s) {
  const int NM = c.N * c.M;
  const size_t smem = smem_taylor(c);
  const int opt = opt_for(NM);
#define AFQ_TAYLOR(K)                                                                          \
  k_taylor<K><<<c.Nw, kThreads, smem, s>>>(phi_io, c.Avhs, c.M, c.N, c.Nw, c.P, c.opt.taylor_order);
  if (opt <= 2) { AFQ_TAYLOR(2) }
  else if (opt <= 4) { AFQ_TAYLOR(4) }
  else if (opt <= 8) { AFQ_TAYLOR(8) }
  else if (opt <= 16) { AFQ_TAYLOR(16) }
  else return cudaErrorInvalidValue;
#undef AFQ_TAYLOR
  return cudaGetLastError();
}

cudaError_t launch_mgs(const Ctx& c, cudaStream_t s) {
  const size_t smem = smem_mgs(c);
  k_mgs<<<c.Nw, 128, smem, s>>>(c.phi, c.alive, c.M, c.N, c.n_up, c.Nw);
  return cudaGetLastError();
}

cudaError_t launch_energy(const Ctx& c, cudaStream_t s, int n_walkers) {
  const size_t smem = smem_energy(c);
  k_energy<<<n_walkers > 0 ? n_walkers : c.Nw, kThreads, smem, s>>>(c.theta, c.Ltil, c.htil, c.eloc, c.M, c.N, c.n_up, c.X, c.Nw);
  return cudaGetLastError();
}

cudaError_t launch_mixed_sum(const Ctx& c, double* out, const int* slot, int slot_stride,
                             cudaStream_t s) {
  k_mixed_sum<<<c.R, 256, 0, s>>>(c.w, c.eloc, out, slot, slot_stride, c.Nw, c.R,
                                  c.opt.mode == AFQMC_FREE);
  return cudaGetLastError();
}

cudaError_t launch_meas_advance(int* meas, cudaStream_t s) {
  k_step_advance<<<1, 32, 0, s>>>(nullptr, meas, 1);
  return cudaGetLastError();
}

cudaError_t launch_step_advance(const Ctx& c, cudaStream_t s) {
  k_step_advance<<<1, 32, 0, s>>>(c.d_step, nullptr, 0);
  return cudaGetLastError();
}

}  // namespace afq
