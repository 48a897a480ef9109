// Reverse-mode (adjoint) kernels of the FP64 propagation step and of the mixed-energy
// measurement, for dE/dh1 along one field realisation.  Complex adjoints follow
// zbar = dL/dRe z + i dL/dIm z; for z = f(u) holomorphic, ubar += zbar conj(f'(u)).
// Layouts: walkers and their adjoints planar [2][Nw][N][M]; per-walker inverses
// Y_s = O_s^{-1} planar [2][Nw][Nup^2 + Ndn^2] (spin-up block first, row-major).
#include <algorithm>
#include <cmath>

#include "device_util.cuh"
#include "internal.h"

namespace afq {
namespace {

constexpr int kT = 256;

// ---------------------------------------------------------------------------
// Inverse overlap per spin, log det and Theta of walkers phi (FP64).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kT) k_inv_overlap(const double* __restrict__ phi,
                                                    const double* __restrict__ psi,
                                                    double* __restrict__ Y, double* __restrict__ logO,
                                                    double* __restrict__ theta,
                                                    const int* __restrict__ mask, int M, int N,
                                                    int n_up, int Nw) {
  extern __shared__ double sm[];
  const int wk = blockIdx.x, tid = threadIdx.x;
  if (mask && !mask[wk]) return;
  const int nmax = max(n_up, N - n_up), nn = n_up * n_up + (N - n_up) * (N - n_up);
  double* ph = sm;                   // [2][nmax][M]
  double* aug = ph + 2 * nmax * M;   // [2][nmax][2 nmax]
  double* fac = aug + 4 * nmax * nmax;
  __shared__ double s_ld[2];
  __shared__ int s_piv, s_bad;
  const int64_t plane = (int64_t)Nw * N * M, wbase = (int64_t)wk * N * M;
  if (tid == 0) { s_ld[0] = s_ld[1] = 0.0; s_bad = 0; }
  for (int sp = 0; sp < 2; ++sp) {
    const int n0 = sp ? n_up : 0, ns = sp ? N - n_up : n_up, yoff = sp ? n_up * n_up : 0;
    if (ns == 0) continue;
    const int w2 = 2 * ns;
    __syncthreads();
    for (int e = tid; e < ns * M; e += blockDim.x) {
      ph[e] = phi[wbase + (int64_t)n0 * M + e];
      ph[nmax * M + e] = phi[plane + wbase + (int64_t)n0 * M + e];
    }
    __syncthreads();
    for (int e = tid; e < ns * w2; e += blockDim.x) {
      const int r = e / w2, c = e % w2;
      double re = 0, im = 0;
      if (c < ns) {
        const double* pr = psi + (int64_t)(n0 + r) * M;
        for (int i = 0; i < M; ++i) {
          re = fma(__ldg(pr + i), ph[c * M + i], re);
          im = fma(__ldg(pr + i), ph[nmax * M + c * M + i], im);
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
        const cplx v = cmul({fac[2 + 2 * r], fac[3 + 2 * r]}, {ar[k * w2 + c], ai[k * w2 + c]});
        ar[e] -= v.re;
        ai[e] -= v.im;
      }
      __syncthreads();
    }
    __syncthreads();
    for (int e = tid; e < ns * ns; e += blockDim.x) {
      const int r = e / ns, c = e % ns;
      Y[(int64_t)wk * nn + yoff + e] = ar[r * w2 + ns + c];
      Y[(int64_t)Nw * nn + (int64_t)wk * nn + yoff + e] = ai[r * w2 + ns + c];
    }
    if (theta)
      for (int e = tid; e < ns * M; e += blockDim.x) {
        const int b = e / M, i = e % M;
        double re = 0, im = 0;
        for (int c = 0; c < ns; ++c) {
          const cplx v = cmul({ph[c * M + i], ph[nmax * M + c * M + i]},
                              {ar[c * w2 + ns + b], ai[c * w2 + ns + b]});
          re += v.re;
          im += v.im;
        }
        theta[wbase + (int64_t)(n0 + b) * M + i] = re;
        theta[plane + wbase + (int64_t)(n0 + b) * M + i] = im;
      }
  }
  __syncthreads();
  if (tid == 0) {
    logO[wk] = s_ld[0];
    logO[Nw + wk] = s_ld[1];
  }
}

// ---------------------------------------------------------------------------
// Rbar = lwbar (1 - i tan theta), theta = Im(log s + log O' - log O), for walkers alive
// after the step; the rest get no adjoint flow (also lwbar and phibar' zeroed).
// ---------------------------------------------------------------------------
__global__ void k_rbar(const double* __restrict__ aux, const double* __restrict__ logO_new,
                       const double* __restrict__ logO_old, const int* __restrict__ still,
                       double* __restrict__ lwbar, double* __restrict__ rbar, int Nw) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Nw) return;
  if (!still[k]) {
    lwbar[k] = 0.0;
    rbar[k] = rbar[Nw + k] = 0.0;
    return;
  }
  const double th = aux[4 * (int64_t)k + 1] + logO_new[Nw + k] - logO_old[Nw + k];
  const double lb = lwbar[k];
  rbar[k] = lb;
  rbar[Nw + k] = -lb * tan(th);
}

__global__ void k_mask_adjoint(double* __restrict__ pb, const int* __restrict__ still, int Nw,
                               int NM) {
  const int64_t total = (int64_t)Nw * NM;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (!still[e / NM]) {
      pb[e] = 0.0;
      pb[total + e] = 0.0;
    }
  }
}

// phibar += sgn * rbar conj(Psi Y^T)  (adjoint of log det(Psi^T Phi) times Rbar)
__global__ void __launch_bounds__(kT) k_logdet_adj(double* __restrict__ pb, const double* __restrict__ psi,
                                                   const double* __restrict__ Y,
                                                   const double* __restrict__ rbar, double sgn,
                                                   int M, int N, int n_up, int Nw) {
  const int wk = blockIdx.x;
  const int nn = n_up * n_up + (N - n_up) * (N - n_up);
  const double rr = rbar[wk] * sgn, ri = rbar[Nw + wk] * sgn;
  if (rr == 0.0 && ri == 0.0) return;
  const int64_t plane = (int64_t)Nw * N * M, wbase = (int64_t)wk * N * M;
  for (int e = threadIdx.x; e < N * M; e += blockDim.x) {
    const int n = e / M, i = e % M;
    const int sp = n < n_up ? 0 : 1, ns = sp ? N - n_up : n_up, n0 = sp ? n_up : 0, b = n - n0;
    const int yoff = sp ? n_up * n_up : 0;
    // (Psi Y^T)[i][b] = sum_a psi[n0+a][i] Y[b][a]
    double gr = 0, gi = 0;
    for (int a = 0; a < ns; ++a) {
      const double p = __ldg(psi + (int64_t)(n0 + a) * M + i);
      gr += p * Y[(int64_t)wk * nn + yoff + b * ns + a];
      gi += p * Y[(int64_t)Nw * nn + (int64_t)wk * nn + yoff + b * ns + a];
    }
    // rbar * conj(g)
    pb[wbase + e] += rr * gr + ri * gi;
    pb[plane + wbase + e] += ri * gr - rr * gi;
  }
}

// ---------------------------------------------------------------------------
// Taylor reverse: recompute T_0 = Phi1, T_n = A T_{n-1}/n (kept in scratch), then
//   Tb = Phibar2; for n = order..1: Abar += Tb T_{n-1}^H / n; Tb = Phibar2 + A^H Tb / n.
// Outputs Phibar1 = Tb (in place of Phibar2), Abar (full M x M, planar), Phi2 = sum T_n.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void packed_mac(const double* ar, const double* ai, int M, int i,
                                           const double* tr, const double* ti, int N, int b,
                                           bool conj_a, double& sr, double& si) {
  const double s = conj_a ? -1.0 : 1.0;
  int64_t rbj = 0;
  for (int j = 0; j < i; ++j) {
    const double xr = __ldg(ar + rbj + i), xi = s * __ldg(ai + rbj + i);
    const double yr = tr[j * N + b], yi = ti[j * N + b];
    sr = fma(xr, yr, fma(-xi, yi, sr));
    si = fma(xr, yi, fma(xi, yr, si));
    rbj += (M - 1) - j;
  }
  const int64_t rbi = (int64_t)i * (M - 1) - (int64_t)i * (i - 1) / 2;
  for (int j = i; j < M; ++j) {
    const double xr = __ldg(ar + rbi + j), xi = s * __ldg(ai + rbi + j);
    const double yr = tr[j * N + b], yi = ti[j * N + b];
    sr = fma(xr, yr, fma(-xi, yi, sr));
    si = fma(xr, yi, fma(xi, yr, si));
  }
}

__global__ void __launch_bounds__(kT) k_taylor_rev(const double* __restrict__ phi1,
                                                   double* __restrict__ pbar,
                                                   const double* __restrict__ Ap,
                                                   double* __restrict__ terms,
                                                   double* __restrict__ Abar,
                                                   double* __restrict__ phi2,
                                                   const int* __restrict__ mask, int M, int N,
                                                   int Nw, int64_t P, int order) {
  extern __shared__ double sm[];
  const int wk = blockIdx.x, tid = threadIdx.x, NM = N * M;
  if (!mask[wk]) {   // no adjoint flows through a walker that did not survive the step
    const int64_t MM = (int64_t)M * M;
    for (int64_t e = tid; e < MM; e += blockDim.x) {
      Abar[(int64_t)wk * MM + e] = 0.0;
      Abar[(int64_t)Nw * MM + (int64_t)wk * MM + e] = 0.0;
    }
    return;
  }
  double* tr = sm;          // working term / adjoint [M][N] layout (row i, column b)
  double* ti = tr + NM;
  double* br = ti + NM;     // Phibar2
  double* bi = br + NM;
  double* nr = bi + NM;
  double* ni = nr + NM;
  const int64_t plane = (int64_t)Nw * NM, base = (int64_t)wk * NM;
  const int64_t tstride = 2 * (int64_t)NM;   // per term per walker in `terms`: [order][Nw][2][NM]
  double* tw = terms + (int64_t)wk * tstride;
  const int64_t tplane = (int64_t)Nw * tstride;
  const double* ar = Ap + (int64_t)wk * P;
  const double* ai = Ap + (int64_t)Nw * P + (int64_t)wk * P;
  for (int o = tid; o < NM; o += blockDim.x) {
    const int i = o / N, b = o % N;
    const int64_t gi = base + (int64_t)b * M + i;
    tr[o] = phi1[gi];
    ti[o] = phi1[plane + gi];
    br[o] = pbar[gi];
    bi[o] = pbar[plane + gi];
  }
  __syncthreads();
  // forward: store T_0 .. T_{order-1}; Phi2 = sum_{n<=order} T_n
  double acc_r[16], acc_i[16];   // up to 16 outputs per thread (N M <= 4096)
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int o = tid + q * kT;
    acc_r[q] = o < NM ? tr[o] : 0.0;
    acc_i[q] = o < NM ? ti[o] : 0.0;
  }
  for (int n = 1; n <= order; ++n) {
    for (int o = tid; o < NM; o += blockDim.x) {
      tw[(int64_t)(n - 1) * tplane + o] = tr[o];
      tw[(int64_t)(n - 1) * tplane + NM + o] = ti[o];
    }
    const double inv = 1.0 / n;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int o = tid + q * kT;
      if (o < NM) {
        const int i = o / N, b = o % N;
        double sr = 0, si = 0;
        packed_mac(ar, ai, M, i, tr, ti, N, b, false, sr, si);
        nr[o] = sr * inv;
        ni[o] = si * inv;
        acc_r[q] += sr * inv;
        acc_i[q] += si * inv;
      }
    }
    __syncthreads();
    for (int o = tid; o < NM; o += blockDim.x) {
      tr[o] = nr[o];
      ti[o] = ni[o];
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int o = tid + q * kT;
    if (o < NM) {
      const int i = o / N, b = o % N;
      const int64_t gi = base + (int64_t)b * M + i;
      phi2[gi] = acc_r[q];
      phi2[plane + gi] = acc_i[q];
    }
  }
  // reverse: Tb (in tr/ti) starts as Phibar2
  for (int o = tid; o < NM; o += blockDim.x) {
    tr[o] = br[o];
    ti[o] = bi[o];
  }
  // Abar accumulated in registers per (i, j) owned by this thread, then stored
  const int MM = M * M;
  double* abr = Abar + (int64_t)wk * MM;
  double* abi = Abar + (int64_t)Nw * MM + (int64_t)wk * MM;
  for (int e = tid; e < MM; e += blockDim.x) {
    abr[e] = 0.0;
    abi[e] = 0.0;
  }
  __syncthreads();
  for (int n = order; n >= 1; --n) {
    const double inv = 1.0 / n;
    const double* Tp = tw + (int64_t)(n - 1) * tplane;   // T_{n-1}
    // Abar[i][j] += sum_b Tb[i][b] conj(T_{n-1}[j][b]) / n
    for (int e = tid; e < MM; e += blockDim.x) {
      const int i = e / M, j = e % M;
      double sr = 0, si = 0;
      for (int b = 0; b < N; ++b) {
        const double xr = tr[i * N + b], xi = ti[i * N + b];
        const double yr = Tp[j * N + b], yi = Tp[NM + j * N + b];
        sr += xr * yr + xi * yi;
        si += xi * yr - xr * yi;
      }
      abr[e] += sr * inv;
      abi[e] += si * inv;
    }
    // Tb <- Phibar2 + A^H Tb / n   (A complex symmetric: A^H = conj(A))
    for (int o = tid; o < NM; o += blockDim.x) {
      const int i = o / N, b = o % N;
      double sr = 0, si = 0;
      packed_mac(ar, ai, M, i, tr, ti, N, b, true, sr, si);
      nr[o] = br[o] + sr * inv;
      ni[o] = bi[o] + si * inv;
    }
    __syncthreads();
    for (int o = tid; o < NM; o += blockDim.x) {
      tr[o] = nr[o];
      ti[o] = ni[o];
    }
    __syncthreads();
  }
  for (int o = tid; o < NM; o += blockDim.x) {
    const int i = o / N, b = o % N;
    const int64_t gi = base + (int64_t)b * M + i;
    pbar[gi] = tr[o];
    pbar[plane + gi] = ti[o];
  }
}

// ---------------------------------------------------------------------------
// Ebar[i][j] += sum_rows Re(X[row][i] conj(Y[row][j])), rows = (walker, orbital) columns.
// X, Y planar [2][rows][M]; each CTA reduces a 32 x 32 tile over one slice of rows into
// its own partial, and k_outer_sum adds the slices in a fixed order (no atomics, so a
// recomputed pass reproduces the sum bit for bit).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_outer_re(const double* __restrict__ Xm, const double* __restrict__ Ym,
                                                  const int* __restrict__ mask, int64_t rows,
                                                  int N, int M, double* __restrict__ part) {
  __shared__ double xs[2][32][33], ys[2][32][33];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  const int64_t per = (rows + gridDim.z - 1) / gridDim.z;
  const int64_t r0 = blockIdx.z * per, r1 = min(rows, r0 + per);
  double acc[4] = {0, 0, 0, 0};
  for (int64_t rb = r0; rb < r1; rb += 32) {
    for (int q = 0; q < 4; ++q) {
      const int rl = ty + 8 * q;
      const int64_t row = rb + rl;
      const bool ok = row < r1 && mask[row / N];
      const int i = i0 + tx, j = j0 + tx;
      xs[0][rl][tx] = (ok && i < M) ? Xm[row * M + i] : 0.0;
      xs[1][rl][tx] = (ok && i < M) ? Xm[rows * M + row * M + i] : 0.0;
      ys[0][rl][tx] = (ok && j < M) ? Ym[row * M + j] : 0.0;
      ys[1][rl][tx] = (ok && j < M) ? Ym[rows * M + row * M + j] : 0.0;
    }
    __syncthreads();
    for (int rl = 0; rl < 32; ++rl) {
      const double a0 = xs[0][rl][tx], a1 = xs[1][rl][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int jl = ty + 8 * q;
        acc[q] += a0 * ys[0][rl][jl] + a1 * ys[1][rl][jl];
      }
    }
    __syncthreads();
  }
  double* pz = part + (int64_t)blockIdx.z * M * M;
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + tx, j = j0 + ty + 8 * q;
    if (i < M && j < M) pz[(int64_t)i * M + j] = acc[q];
  }
}

__global__ void k_outer_sum(const double* __restrict__ part, int nz, int MM, double* __restrict__ Ebar) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= MM) return;
  double s = Ebar[e];
  for (int z = 0; z < nz; ++z) s += part[(int64_t)z * MM + e];
  Ebar[e] = s;
}

// ---------------------------------------------------------------------------
// Fields reverse: from S = sum_ij L_g,ij Abar_ij (planar [2][Nw][X]), Rbar and lwbar:
//   cbar_g = conj(i sqrt(dt)) S_g + Rbar conj(-i sqrt(dt) <rho_g>)
//   xbarbar = lwbar conj(x - xbar) - cbar; through the cap; rhobarbar = conj(-i sqrt(dt)) x_rbar
// ---------------------------------------------------------------------------
struct FieldRevArgs {
  const double *rhobar, *rho_mf, *fields, *S, *rbar, *lwbar;
  double* rbb;   // [2][Nw][X]
  const int* mask;
  const unsigned long long* step;
  uint2 key;
  uint32_t k0;
  int X, Nw;
  double sqrt_dt, fb_cap;
};

__global__ void __launch_bounds__(128) k_fields_rev(FieldRevArgs a) {
  const int wk = blockIdx.x, X = a.X;
  const uint32_t t = (uint32_t)(*a.step);
  const int64_t row = (int64_t)wk * X, plane = (int64_t)a.Nw * X;
  if (!a.mask[wk]) {
    for (int g = threadIdx.x; g < X; g += blockDim.x) a.rbb[row + g] = a.rbb[plane + row + g] = 0.0;
    return;
  }
  const double Rr = a.rbar[wk], Ri = a.rbar[a.Nw + wk], lb = a.lwbar[wk];
  for (int j = threadIdx.x; j < (X + 1) / 2; j += blockDim.x) {
    double z[2];
    if (a.fields == nullptr) {
      const uint4 r = philox4x32_10(make_uint4((uint32_t)j, a.k0 + (uint32_t)wk, t, 0u), a.key);
      philox_normal2(r, z[0], z[1]);
    }
    for (int q = 0; q < 2; ++q) {
      const int g = 2 * j + q;
      if (g >= X) break;
      const double x = a.fields ? a.fields[row + g] : z[q];
      const double xr0 = a.sqrt_dt * a.rhobar[plane + row + g];
      const double xi0 = -a.sqrt_dt * (a.rhobar[row + g] - a.rho_mf[g]);
      double xbr = xr0, xbi = xi0;
      bool capped = false;
      double m = 0;
      if (a.fb_cap > 0.0) {
        const double m2 = xr0 * xr0 + xi0 * xi0;
        if (m2 > a.fb_cap * a.fb_cap) {
          capped = true;
          m = sqrt(m2);
          xbr *= a.fb_cap / m;
          xbi *= a.fb_cap / m;
        }
      }
      // cbar: conj(i sqrt(dt)) S = -i sqrt(dt) (S_re + i S_im) = sqrt(dt) S_im - i sqrt(dt) S_re
      const double Sr = a.S[row + g], Si = a.S[plane + row + g];
      double cbr = a.sqrt_dt * Si, cbi = -a.sqrt_dt * Sr;
      // + Rbar conj(-i sqrt(dt) rho) = Rbar (i sqrt(dt) rho)
      const double rm = a.rho_mf[g];
      cbr += -Ri * a.sqrt_dt * rm;
      cbi += Rr * a.sqrt_dt * rm;
      // xbarbar = lwbar conj(x - xbar) - cbar
      double ur = lb * (x - xbr) - cbr, ui = lb * xbi - cbi;
      if (capped) {
        // zbar = (cap/|z|) (ubar - Re(conj(ubar) z) z / |z|^2)
        const double proj = (ur * xr0 + ui * xi0) / (m * m);
        const double sc = a.fb_cap / m;
        ur = sc * (ur - proj * xr0);
        ui = sc * (ui - proj * xi0);
      }
      // rhobarbar = conj(-i sqrt(dt)) x_rbar = i sqrt(dt) (ur + i ui)
      a.rbb[row + g] = -a.sqrt_dt * ui;
      a.rbb[plane + row + g] = a.sqrt_dt * ur;
    }
  }
}

// ---------------------------------------------------------------------------
// Overlap reverse at walkers phi with inverses Y:
//   Phibar += Thetabar Y^H + Psi Obar,  Obar = -Y^H (Phi^H Thetabar) Y^H
// (Theta = Phi Y, Y = O^{-1}, O = Psi^T Phi), all per spin.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kT) k_overlap_rev(const double* __restrict__ phi,
                                                    const double* __restrict__ Y,
                                                    const double* __restrict__ thb,
                                                    const double* __restrict__ psi,
                                                    double* __restrict__ pb,
                                                    const int* __restrict__ mask, int M, int N,
                                                    int n_up, int Nw) {
  extern __shared__ double sm[];
  const int wk = blockIdx.x, tid = threadIdx.x;
  if (!mask[wk]) return;
  const int nn = n_up * n_up + (N - n_up) * (N - n_up);
  const int nmax = max(n_up, N - n_up);
  double* yb = sm;                    // Ybar [2][nmax][nmax]
  double* ob = yb + 2 * nmax * nmax;  // Obar [2][nmax][nmax]
  const int64_t plane = (int64_t)Nw * N * M, wbase = (int64_t)wk * N * M;
  const double* yr = Y + (int64_t)wk * nn;
  const double* yi = Y + (int64_t)Nw * nn + (int64_t)wk * nn;
  for (int sp = 0; sp < 2; ++sp) {
    const int n0 = sp ? n_up : 0, ns = sp ? N - n_up : n_up, yoff = sp ? n_up * n_up : 0;
    if (ns == 0) continue;
    __syncthreads();
    // Ybar[c][b] = sum_i conj(Phi[i][c]) Thetabar[i][b]
    for (int e = tid; e < ns * ns; e += blockDim.x) {
      const int c = e / ns, b = e % ns;
      double sr = 0, si = 0;
      for (int i = 0; i < M; ++i) {
        const int64_t gc = wbase + (int64_t)(n0 + c) * M + i, gb = wbase + (int64_t)(n0 + b) * M + i;
        const double pr_ = phi[gc], pi_ = -phi[plane + gc];
        const double tr_ = thb[gb], ti_ = thb[plane + gb];
        sr += pr_ * tr_ - pi_ * ti_;
        si += pr_ * ti_ + pi_ * tr_;
      }
      yb[e] = sr;
      yb[nmax * nmax + e] = si;
    }
    __syncthreads();
    // Obar = -Y^H Ybar Y^H  -> first Z = Ybar Y^H, then Obar = -Y^H Z
    for (int e = tid; e < ns * ns; e += blockDim.x) {
      const int r = e / ns, c = e % ns;
      double sr = 0, si = 0;
      for (int q = 0; q < ns; ++q) {   // Z[r][c] = sum_q Ybar[r][q] conj(Y[c][q])
        const double ar_ = yb[r * ns + q], ai_ = yb[nmax * nmax + r * ns + q];
        const double br_ = yr[yoff + c * ns + q], bi_ = -yi[yoff + c * ns + q];
        sr += ar_ * br_ - ai_ * bi_;
        si += ar_ * bi_ + ai_ * br_;
      }
      ob[e] = sr;
      ob[nmax * nmax + e] = si;
    }
    __syncthreads();
    for (int e = tid; e < ns * ns; e += blockDim.x) {
      const int r = e / ns, c = e % ns;
      double sr = 0, si = 0;
      for (int q = 0; q < ns; ++q) {   // W[r][c] = -sum_q conj(Y[q][r]) Z[q][c]
        const double ar_ = yr[yoff + q * ns + r], ai_ = -yi[yoff + q * ns + r];
        const double br_ = ob[q * ns + c], bi_ = ob[nmax * nmax + q * ns + c];
        sr -= ar_ * br_ - ai_ * bi_;
        si -= ar_ * bi_ + ai_ * br_;
      }
      yb[e] = sr;   // reuse as Obar
      yb[nmax * nmax + e] = si;
    }
    __syncthreads();
    // Phibar[i][b] += sum_c Thetabar[i][c] conj(Y[b][c]) + sum_a psi[n0+a][i] Obar[a][b]
    for (int e = tid; e < ns * M; e += blockDim.x) {
      const int b = e / M, i = e % M;
      double sr = 0, si = 0;
      for (int c = 0; c < ns; ++c) {
        const int64_t gc = wbase + (int64_t)(n0 + c) * M + i;
        const double tr_ = thb[gc], ti_ = thb[plane + gc];
        const double br_ = yr[yoff + b * ns + c], bi_ = -yi[yoff + b * ns + c];
        sr += tr_ * br_ - ti_ * bi_;
        si += tr_ * bi_ + ti_ * br_;
      }
      for (int a = 0; a < ns; ++a) {
        const double p = __ldg(psi + (int64_t)(n0 + a) * M + i);
        sr += p * yb[a * ns + b];
        si += p * yb[nmax * nmax + a * ns + b];
      }
      const int64_t gi = wbase + (int64_t)(n0 + b) * M + i;
      pb[gi] += sr;
      pb[plane + gi] += si;
    }
  }
}

// ---------------------------------------------------------------------------
// Gram-Schmidt reverse: Q = Phi3 R^{-1} with R = Q^H Phi3 (upper triangular, per spin):
//   Phibar_pre = Phibar_post R^{-H}   (solve X R^H = B column by column, from the last).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_mgs_rev(const double* __restrict__ Q, const double* __restrict__ phi3,
                                                 double* __restrict__ pb, const int* __restrict__ alive,
                                                 int M, int N, int n_up, int Nw) {
  __shared__ double R[2][32 * 32];
  __shared__ double red[4 * 4 + 4];
  const int wk = blockIdx.x, tid = threadIdx.x;
  if (!alive[wk]) return;
  const int64_t plane = (int64_t)Nw * N * M, wbase = (int64_t)wk * N * M;
  for (int sp = 0; sp < 2; ++sp) {
    const int n0 = sp ? n_up : 0, ns = sp ? N - n_up : n_up;
    if (ns == 0) continue;
    // R[a][b] = sum_i conj(Q[i][a]) Phi3[i][b]
    for (int e = 0; e < ns * ns; ++e) {
      const int a_ = e / ns, b = e % ns;
      double s[2] = {0, 0};
      for (int i = tid; i < M; i += blockDim.x) {
        const int64_t qa = wbase + (int64_t)(n0 + a_) * M + i, pbx = wbase + (int64_t)(n0 + b) * M + i;
        const double qr = Q[qa], qi = -Q[plane + qa], xr = phi3[pbx], xi = phi3[plane + pbx];
        s[0] += qr * xr - qi * xi;
        s[1] += qr * xi + qi * xr;
      }
      block_allsum<2>(s, red);
      if (tid == 0) { R[0][e] = s[0]; R[1][e] = s[1]; }
    }
    __syncthreads();
    // X[:, j] = (B[:, j] - sum_{k>j} X[:, k] conj(R[j][k])) / conj(R[j][j]), j = ns-1 .. 0
    for (int i = tid; i < M; i += blockDim.x) {
      for (int j = ns - 1; j >= 0; --j) {
        const int64_t gj = wbase + (int64_t)(n0 + j) * M + i;
        double br = pb[gj], bi = pb[plane + gj];
        for (int k = j + 1; k < ns; ++k) {
          const int64_t gk = wbase + (int64_t)(n0 + k) * M + i;
          const double xr = pb[gk], xi = pb[plane + gk];
          const double rr = R[0][j * ns + k], ri = -R[1][j * ns + k];
          br -= xr * rr - xi * ri;
          bi -= xr * ri + xi * rr;
        }
        const cplx d = cinv({R[0][j * ns + j], -R[1][j * ns + j]});
        const cplx v = cmul({br, bi}, d);
        pb[gj] = v.re;
        pb[plane + gj] = v.im;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Measurement reverse: Thetabar of ebar_k Re E_L,k through the half-rotated tensors,
//   Thetabar_s = ebar conj(F_s) Psi_s with
//   [conj(F) Psi][i][a] = htil[a][i] + sum_g conj(rhobar_g) Ltil_g[a][i]
//                         - sum_g sum_b Ltil_g[b][i] conj(T_g[a][b]),  T_g = Ltil_g Theta_s,
// where F = h1 + sum_g rhobar_g L_g - sum_g L_g G L_g = dE_L/dG^T.  Also writes Re E_L.
// ---------------------------------------------------------------------------
constexpr int G_CH = 4;
__global__ void __launch_bounds__(kT) k_energy_rev(const double* __restrict__ theta,
                                                   const double* __restrict__ Ltil,
                                                   const double* __restrict__ htil,
                                                   const double* __restrict__ ebar,
                                                   double* __restrict__ thb, double* __restrict__ eloc,
                                                   const int* __restrict__ mask, int M, int N,
                                                   int n_up, int X, int Nw) {
  extern __shared__ double sm[];
  const int wk = blockIdx.x, tid = threadIdx.x, NM = N * M;
  const int nu = n_up, nd = N - n_up, nn = nu * nu + nd * nd;
  const int64_t plane = (int64_t)Nw * NM, base = (int64_t)wk * NM;
  if (!mask[wk]) {
    for (int e = tid; e < NM; e += blockDim.x) thb[base + e] = thb[plane + base + e] = 0.0;
    if (tid == 0) eloc[wk] = 0.0;
    return;
  }
  double* thr = sm;             // Theta [M][N]
  double* thi = thr + NM;
  double* gr = thi + NM;        // conj(F) Psi accumulators, same layout as the walkers
  double* gi = gr + NM;
  double* Tr = gi + NM;         // [G_CH][nn]
  double* Ti = Tr + G_CH * nn;
  double* cr = Ti + G_CH * nn;  // rhobar_g of the chunk [G_CH][2]
  double* red = cr + 2 * G_CH;
  const double eb = ebar[wk];
  double acc[2] = {0, 0};
  for (int e = tid; e < NM; e += blockDim.x) {
    const int n = e / M, i = e % M;
    const double vr = theta[base + e], vi = theta[plane + base + e];
    thr[i * N + n] = vr;
    thi[i * N + n] = vi;
    const double h = __ldg(htil + e);
    gr[e] = h;
    gi[e] = 0.0;
    acc[0] = fma(h, vr, acc[0]);
    acc[1] = fma(h, vi, acc[1]);
  }
  __syncthreads();
  for (int g0 = 0; g0 < X; g0 += G_CH) {
    const int gc = min(G_CH, X - g0);
    for (int e = tid; e < gc * nn; e += blockDim.x) {
      const int gl = e / nn, r = e % nn;
      int a_, b, n0;
      if (r < nu * nu) { a_ = r / nu; b = r % nu; n0 = 0; }
      else { const int r2 = r - nu * nu; a_ = r2 / nd; b = r2 % nd; n0 = nu; }
      const double* lrow = Ltil + ((int64_t)(g0 + gl) * N + n0 + a_) * M;
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
    for (int gl = tid; gl < gc; gl += blockDim.x) {
      double c0 = 0, c1 = 0;
      for (int a_ = 0; a_ < nu; ++a_) { c0 += Tr[gl * nn + a_ * nu + a_]; c1 += Ti[gl * nn + a_ * nu + a_]; }
      for (int a_ = 0; a_ < nd; ++a_) {
        c0 += Tr[gl * nn + nu * nu + a_ * nd + a_];
        c1 += Ti[gl * nn + nu * nu + a_ * nd + a_];
      }
      cr[2 * gl] = c0;
      cr[2 * gl + 1] = c1;
      acc[0] += 0.5 * (c0 * c0 - c1 * c1);
      acc[1] += c0 * c1;
    }
    for (int e = tid; e < gc * nn; e += blockDim.x) {
      const int gl = e / nn, r = e % nn;
      int et;
      if (r < nu * nu) { const int a_ = r / nu, b = r % nu; et = b * nu + a_; }
      else { const int r2 = r - nu * nu; const int a_ = r2 / nd, b = r2 % nd; et = nu * nu + b * nd + a_; }
      const cplx p = cmul({Tr[e], Ti[e]}, {Tr[gl * nn + et], Ti[gl * nn + et]});
      acc[0] -= 0.5 * p.re;
      acc[1] -= 0.5 * p.im;
    }
    __syncthreads();
    for (int e = tid; e < NM; e += blockDim.x) {
      const int n = e / M, i = e % M;
      const int sp = n < nu ? 0 : 1, ns = sp ? nd : nu, n0 = sp ? nu : 0, a_ = n - n0;
      const int off = sp ? nu * nu : 0;
      double sr = 0, si = 0;
      for (int gl = 0; gl < gc; ++gl) {
        const double* lg = Ltil + (int64_t)(g0 + gl) * NM;
        const double la = __ldg(lg + (int64_t)(n0 + a_) * M + i);
        sr += cr[2 * gl] * la;
        si -= cr[2 * gl + 1] * la;
        for (int b = 0; b < ns; ++b) {
          const double l = __ldg(lg + (int64_t)(n0 + b) * M + i);
          const int q = gl * nn + off + a_ * ns + b;
          sr -= l * Tr[q];
          si += l * Ti[q];
        }
      }
      gr[e] += sr;
      gi[e] += si;
    }
    __syncthreads();
  }
  for (int e = tid; e < NM; e += blockDim.x) {
    thb[base + e] = eb * gr[e];
    thb[plane + base + e] = eb * gi[e];
  }
  block_sum<2>(acc, red);
  if (tid == 0) eloc[wk] = acc[0];
}

// ebar_k = w_k / (sum_alive w n_meas) for live walkers, 0 otherwise (one CTA).
__global__ void __launch_bounds__(256) k_meas_weights(const double* __restrict__ w, const int* __restrict__ alive,
                                                      double* __restrict__ ebar, int Nw, double inv_meas) {
  __shared__ double red[4 * 8 + 4];
  double v[1] = {0.0};
  for (int k = threadIdx.x; k < Nw; k += blockDim.x) v[0] += alive[k] ? w[k] : 0.0;
  block_allsum<1>(v, red);
  const double W = v[0];
  for (int k = threadIdx.x; k < Nw; k += blockDim.x)
    ebar[k] = (alive[k] && W > 0.0) ? w[k] / W * inv_meas : 0.0;
}

// E_m = n_meas sum_k ebar_k Re E_L,k;  E += E_m / n_meas;  lwbar_k += ebar_k (E_L,k - E_m)
// (d E_m / d log w_k = w_k (E_L,k - E_m) / W).  NaN into E when no walker is alive.  One CTA.
__global__ void __launch_bounds__(256) k_meas_finish(const double* __restrict__ eloc, const double* __restrict__ ebar,
                                                     double* __restrict__ lwbar, double* __restrict__ e_acc,
                                                     int Nw, double n_meas) {
  __shared__ double red[4 * 8 + 4];
  double v[2] = {0.0, 0.0};
  for (int k = threadIdx.x; k < Nw; k += blockDim.x) {
    if (ebar[k] == 0.0) continue;   // dead walker: its E_L need not be finite
    v[0] += ebar[k] * eloc[k];
    v[1] += ebar[k];
  }
  block_allsum<2>(v, red);
  const double Em = v[0] * n_meas;
  for (int k = threadIdx.x; k < Nw; k += blockDim.x)
    if (ebar[k] != 0.0) lwbar[k] += ebar[k] * (eloc[k] - Em);
  if (threadIdx.x == 0) *e_acc += v[1] > 0.0 ? Em / n_meas : NAN;
}

// avg[n][i] += sum_k ebar_k Re Theta_k[n][i]   (the direct one-body term of E_L)
__global__ void k_theta_avg(const double* __restrict__ theta, const double* __restrict__ ebar,
                            double* __restrict__ avg, int Nw, int NM) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NM) return;
  double s = 0;
  for (int k = 0; k < Nw; ++k) {
    const double eb = ebar[k];
    if (eb != 0.0) s += eb * theta[(int64_t)k * NM + e];
  }
  avg[e] += s;
}

// out[i][j] = alpha L[i][j] + sum_n avg[n][i] psi[n][j]   (h1bar = -dt/2 L_exp(B, Ebar) +
// sum_k ebar_k Re G_k^T, G = Psi Theta^T per spin)
__global__ void k_h1bar(const double* __restrict__ Lx, double alpha, const double* __restrict__ avg,
                        const double* __restrict__ psi, double* __restrict__ out, int M, int N) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * M) return;
  const int i = e / M, j = e % M;
  double s = alpha * Lx[e];
  for (int n = 0; n < N; ++n) s += avg[n * M + i] * psi[n * M + j];
  out[e] = s;
}

// Z[(r0 + r) * ldz + c0 + c] = alpha * src[r * M + c]
__global__ void k_place_block(double* __restrict__ Z, int ldz, int r0, int c0,
                              const double* __restrict__ src, int M, double alpha) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * M) return;
  const int r = e / M, c = e % M;
  Z[(int64_t)(r0 + r) * ldz + c0 + c] = alpha * src[e];
}

// dst[r * M + c] = alpha * Z[(r0 + r) * ldz + c0 + c]
__global__ void k_take_block(const double* __restrict__ Z, int ldz, int r0, int c0,
                             double* __restrict__ dst, int M, double alpha) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * M) return;
  const int r = e / M, c = e % M;
  dst[e] = alpha * Z[(int64_t)(r0 + r) * ldz + c0 + c];
}

__global__ void k_set_step(unsigned long long* step, unsigned long long v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *step = v;
}

}  // namespace

size_t smem_inv_overlap(const Ctx& c) {
  const size_t nmax = c.n_up > c.N - c.n_up ? c.n_up : c.N - c.n_up;
  return sizeof(double) * (2 * nmax * c.M + 4 * nmax * nmax + 2 * nmax + 2);
}
size_t smem_taylor_rev(const Ctx& c) { return sizeof(double) * 6 * (size_t)c.N * c.M; }
size_t smem_overlap_rev(const Ctx& c) {
  const size_t nmax = c.n_up > c.N - c.n_up ? c.n_up : c.N - c.n_up;
  return sizeof(double) * 4 * nmax * nmax;
}
size_t smem_energy_rev(const Ctx& c) {
  const size_t nu = c.n_up, nd = c.N - c.n_up, nn = nu * nu + nd * nd;
  return sizeof(double) * (4 * (size_t)c.N * c.M + 2 * G_CH * nn + 2 * G_CH + 64);
}

bool adjoint_fits(const Ctx& c) {
  return smem_taylor_rev(c) <= 200 * 1024 && smem_energy_rev(c) <= 200 * 1024 &&
         smem_inv_overlap(c) <= 200 * 1024 && (size_t)c.N * c.M <= 16 * kT && c.n_up <= 32 &&
         c.N - c.n_up <= 32;
}

cudaError_t prepare_adjoint_kernels(const Ctx& c) {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_inv_overlap, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_inv_overlap(c))) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_taylor_rev, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_taylor_rev(c))) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_overlap_rev, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_overlap_rev(c))) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_energy_rev, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_energy_rev(c));
}

cudaError_t adj_inv_overlap(const Ctx& c, const double* phi, double* Y, double* logO, double* theta,
                            const int* mask, cudaStream_t s) {
  k_inv_overlap<<<c.Nw, kT, smem_inv_overlap(c), s>>>(phi, c.psi, Y, logO, theta, mask, c.M, c.N,
                                                      c.n_up, c.Nw);
  return cudaGetLastError();
}
cudaError_t adj_rbar(const Ctx& c, const double* logO_new, const double* logO_old, const int* still,
                     double* lwbar, double* rbar, cudaStream_t s) {
  k_rbar<<<(c.Nw + 255) / 256, 256, 0, s>>>(c.aux, logO_new, logO_old, still, lwbar, rbar, c.Nw);
  return cudaGetLastError();
}
cudaError_t adj_mask(const Ctx& c, double* pb, const int* still, cudaStream_t s) {
  const int64_t n = (int64_t)c.Nw * c.N * c.M;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  k_mask_adjoint<<<grid < 1 ? 1 : grid, 256, 0, s>>>(pb, still, c.Nw, c.N * c.M);
  return cudaGetLastError();
}
cudaError_t adj_logdet(const Ctx& c, double* pb, const double* Y, const double* rbar, double sgn,
                       cudaStream_t s) {
  k_logdet_adj<<<c.Nw, kT, 0, s>>>(pb, c.psi, Y, rbar, sgn, c.M, c.N, c.n_up, c.Nw);
  return cudaGetLastError();
}
cudaError_t adj_taylor(const Ctx& c, const double* phi1, double* pbar, double* terms, double* Abar,
                       double* phi2, const int* mask, cudaStream_t s) {
  k_taylor_rev<<<c.Nw, kT, smem_taylor_rev(c), s>>>(phi1, pbar, c.Avhs, terms, Abar, phi2, mask, c.M,
                                                    c.N, c.Nw, c.P, c.opt.taylor_order);
  return cudaGetLastError();
}
cudaError_t adj_outer(const Ctx& c, const double* Xm, const double* Ym, const int* mask, double* part,
                      double* Ebar, cudaStream_t s) {
  const int64_t rows = (int64_t)c.Nw * c.N;
  const int tiles = ((c.M + 31) / 32) * ((c.M + 31) / 32);
  int zs = (int)std::min<int64_t>((rows + 31) / 32, std::max(1, 2 * 152 / tiles));
  zs = std::max(1, std::min(zs, kOuterSlices));
  dim3 grid((c.M + 31) / 32, (c.M + 31) / 32, zs);
  k_outer_re<<<grid, 256, 0, s>>>(Xm, Ym, mask, rows, c.N, c.M, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int MM = c.M * c.M;
  k_outer_sum<<<(MM + 255) / 256, 256, 0, s>>>(part, zs, MM, Ebar);
  return cudaGetLastError();
}
cudaError_t adj_fields(const Ctx& c, const double* fields, const double* S, const double* rbar,
                       const double* lwbar, double* rbb, const int* mask, cudaStream_t s) {
  FieldRevArgs a;
  a.rhobar = c.rhobar; a.rho_mf = c.rho_mf; a.fields = fields; a.S = S; a.rbar = rbar;
  a.lwbar = lwbar; a.rbb = rbb; a.mask = mask; a.step = c.d_step;
  a.key = make_uint2((uint32_t)(c.opt.seed & 0xffffffffull), (uint32_t)(c.opt.seed >> 32));
  a.k0 = (uint32_t)c.opt.walker_offset;
  a.X = c.X; a.Nw = c.Nw; a.sqrt_dt = c.sqrt_dt; a.fb_cap = c.opt.fb_cap;
  k_fields_rev<<<c.Nw, 128, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t adj_overlap(const Ctx& c, const double* phi, const double* Y, const double* thb,
                        double* pb, const int* mask, cudaStream_t s) {
  k_overlap_rev<<<c.Nw, kT, smem_overlap_rev(c), s>>>(phi, Y, thb, c.psi, pb, mask, c.M, c.N, c.n_up,
                                                      c.Nw);
  return cudaGetLastError();
}
cudaError_t adj_mgs(const Ctx& c, const double* Q, const double* phi3, double* pb, const int* alive,
                    cudaStream_t s) {
  k_mgs_rev<<<c.Nw, 128, 0, s>>>(Q, phi3, pb, alive, c.M, c.N, c.n_up, c.Nw);
  return cudaGetLastError();
}
cudaError_t adj_energy(const Ctx& c, const double* theta, const double* ebar, double* thb,
                       double* eloc, const int* mask, cudaStream_t s) {
  k_energy_rev<<<c.Nw, kT, smem_energy_rev(c), s>>>(theta, c.Ltil, c.htil, ebar, thb, eloc, mask, c.M,
                                                    c.N, c.n_up, c.X, c.Nw);
  return cudaGetLastError();
}
cudaError_t adj_meas_weights(const Ctx& c, double* ebar, double inv_meas, cudaStream_t s) {
  k_meas_weights<<<1, 256, 0, s>>>(c.w, c.alive, ebar, c.Nw, inv_meas);
  return cudaGetLastError();
}
cudaError_t adj_meas_finish(const Ctx& c, const double* eloc, const double* ebar, double* lwbar,
                            double* e_acc, double n_meas, cudaStream_t s) {
  k_meas_finish<<<1, 256, 0, s>>>(eloc, ebar, lwbar, e_acc, c.Nw, n_meas);
  return cudaGetLastError();
}
cudaError_t adj_theta_avg(const Ctx& c, const double* theta, const double* ebar, double* avg,
                          cudaStream_t s) {
  const int NM = c.N * c.M;
  k_theta_avg<<<(NM + 255) / 256, 256, 0, s>>>(theta, ebar, avg, c.Nw, NM);
  return cudaGetLastError();
}
cudaError_t adj_h1bar(const Ctx& c, const double* Lx, double alpha, const double* avg, double* out,
                      cudaStream_t s) {
  const int MM = c.M * c.M;
  k_h1bar<<<(MM + 255) / 256, 256, 0, s>>>(Lx, alpha, avg, c.psi, out, c.M, c.N);
  return cudaGetLastError();
}
cudaError_t place_block(double* Z, int ldz, int r0, int c0, const double* src, int M, double alpha,
                        cudaStream_t s) {
  k_place_block<<<(M * M + 255) / 256, 256, 0, s>>>(Z, ldz, r0, c0, src, M, alpha);
  return cudaGetLastError();
}
cudaError_t take_block(const double* Z, int ldz, int r0, int c0, double* dst, int M, double alpha,
                       cudaStream_t s) {
  k_take_block<<<(M * M + 255) / 256, 256, 0, s>>>(Z, ldz, r0, c0, dst, M, alpha);
  return cudaGetLastError();
}
cudaError_t set_step(const Ctx& c, unsigned long long v, cudaStream_t s) {
  k_set_step<<<1, 32, 0, s>>>(c.d_step, v);
  return cudaGetLastError();
}

}  // namespace afq
