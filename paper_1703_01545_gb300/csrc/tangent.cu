// Tangent-mode (forward) derivative of the propagation and the mixed energy along a one-body
// perturbation h1 -> h1 + lambda P, with the fields and the trial held fixed (FP64 path).
//
// Every walker carries dPhi (same layout as Phi) and d log w.  Per step:
//   drhobar = Ltil . dTheta            (force-bias GEMM on the tangent of Theta)
//   dxbar = -i sqrt(dt) drhobar (through the cap), dc = -dxbar, dU = i sqrt(dt) dc
//   dA = sum_g dU_g L_g                 (V_HS GEMM on dU)
//   dPhi1 = dE Phi + E dPhi;  dT_n = (dA T_{n-1} + A dT_{n-1}) / n;  dPhi' = dE Phi2 + E dPhi2
//   dlog O = sum_s tr(O_s^{-1} Psi_s^T dPhi_s),  dTheta_s = (dPhi_s - Theta_s Psi_s^T dPhi_s) O_s^{-1}
//   dlog I = dlog s + dlog O' - dlog O + (x - xbar).dxbar + dt dE_T
//   dlog w += Re dlog I - tan(arg R) Im(dlog s + dlog O' - dlog O)        (while cos > 0)
// MGS applies the same column operations to dPhi (dPhi R^{-1}).  E is exp(-dt K/2); dE is
// its Frechet derivative along -dt P/2.
#include <cmath>

#include "device_util.cuh"
#include "internal.h"

namespace afq {
namespace {

constexpr int kT = 256;

// ---- fields with tangents ----
struct FieldTanArgs {
  const double *rhobar, *drhobar, *rho_mf, *fields;
  double *U, *dU, *aux, *daux;
  const unsigned long long* step;
  uint2 key;
  uint32_t k0;
  int X, Nw;
  double sqrt_dt, fb_cap;
};

__global__ void __launch_bounds__(128) k_fields_tan(FieldTanArgs a) {
  __shared__ double red[4 * 4 + 4];
  const int wk = blockIdx.x, X = a.X;
  const uint32_t t = (uint32_t)(*a.step);
  const int64_t row = (int64_t)wk * X, plane = (int64_t)a.Nw * X;
  double acc[4] = {0, 0, 0, 0}, dacc[4] = {0, 0, 0, 0};
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
      double xr = a.sqrt_dt * a.rhobar[plane + row + g];
      double xi = -a.sqrt_dt * (a.rhobar[row + g] - a.rho_mf[g]);
      double dxr = a.sqrt_dt * a.drhobar[plane + row + g];
      double dxi = -a.sqrt_dt * a.drhobar[row + g];
      if (a.fb_cap > 0.0) {
        const double m2 = xr * xr + xi * xi;
        if (m2 > a.fb_cap * a.fb_cap) {
          const double m = sqrt(m2), sc = a.fb_cap / m;
          const double proj = (xr * dxr + xi * dxi) / m2;   // Re(conj(x) dx) / |x|^2
          dxr = sc * (dxr - xr * proj);
          dxi = sc * (dxi - xi * proj);
          xr *= sc;
          xi *= sc;
        }
      }
      const double cr = x - xr, ci = -xi, dcr = -dxr, dci = -dxi;
      a.U[row + g] = -a.sqrt_dt * ci;
      a.U[plane + row + g] = a.sqrt_dt * cr;
      a.dU[row + g] = -a.sqrt_dt * dci;
      a.dU[plane + row + g] = a.sqrt_dt * dcr;
      const double rm = a.rho_mf[g];
      acc[0] = fma(cr, rm, acc[0]);
      acc[1] = fma(ci, rm, acc[1]);
      acc[2] += x * xr - 0.5 * (xr * xr - xi * xi);
      acc[3] += x * xi - xr * xi;
      dacc[0] = fma(dcr, rm, dacc[0]);
      dacc[1] = fma(dci, rm, dacc[1]);
      // d(x.xbar - xbar^2/2) = (x - xbar) dxbar (complex)
      dacc[2] += (x - xr) * dxr + xi * dxi;
      dacc[3] += (x - xr) * dxi - xi * dxr;
    }
  }
  block_sum<4>(acc, red);
  if (threadIdx.x == 0) {
    double* o = a.aux + 4 * (int64_t)wk;
    o[0] = a.sqrt_dt * acc[1];
    o[1] = -a.sqrt_dt * acc[0];
    o[2] = acc[2];
    o[3] = acc[3];
  }
  __syncthreads();
  block_sum<4>(dacc, red);
  if (threadIdx.x == 0) {
    double* o = a.daux + 4 * (int64_t)wk;
    o[0] = a.sqrt_dt * dacc[1];
    o[1] = -a.sqrt_dt * dacc[0];
    o[2] = dacc[2];
    o[3] = dacc[3];
  }
}

// ---- Taylor exponential with tangent: phi, dphi in place (FP64), A, dA packed ----
__device__ __forceinline__ void packed_row_mac(const double* ar, const double* ai, int M, int i,
                                               const double* tr, const double* ti, int N, int b,
                                               double& sr, double& si) {
  int64_t rbj = 0;
  for (int j = 0; j < i; ++j) {
    const double xr = __ldg(ar + rbj + i), xi = __ldg(ai + rbj + i);
    const double yr = tr[j * N + b], yi = ti[j * N + b];
    sr = fma(xr, yr, fma(-xi, yi, sr));
    si = fma(xr, yi, fma(xi, yr, si));
    rbj += (M - 1) - j;
  }
  const int64_t rbi = (int64_t)i * (M - 1) - (int64_t)i * (i - 1) / 2;
  for (int j = i; j < M; ++j) {
    const double xr = __ldg(ar + rbi + j), xi = __ldg(ai + rbi + j);
    const double yr = tr[j * N + b], yi = ti[j * N + b];
    sr = fma(xr, yr, fma(-xi, yi, sr));
    si = fma(xr, yi, fma(xi, yr, si));
  }
}

__global__ void __launch_bounds__(kT) k_taylor_tan(double* __restrict__ phi, double* __restrict__ dphi,
                                                   const double* __restrict__ Ap,
                                                   const double* __restrict__ dAp, int M, int N,
                                                   int Nw, int64_t P, int order) {
  extern __shared__ double sm[];
  const int wk = blockIdx.x, tid = threadIdx.x, NM = N * M;
  double* tr = sm;        // current term
  double* ti = tr + NM;
  double* ur = ti + NM;   // current tangent term
  double* ui = ur + NM;
  double* nr = ui + NM;   // next term
  double* ni = nr + NM;
  double* vr = ni + NM;   // next tangent term
  double* vi = vr + NM;
  const int64_t plane = (int64_t)Nw * NM, base = (int64_t)wk * NM;
  const double* ar = Ap + (int64_t)wk * P;
  const double* ai = Ap + (int64_t)Nw * P + (int64_t)wk * P;
  const double* dar = dAp + (int64_t)wk * P;
  const double* dai = dAp + (int64_t)Nw * P + (int64_t)wk * P;
  for (int o = tid; o < NM; o += blockDim.x) {
    const int i = o / N, b = o % N;
    const int64_t gi = base + (int64_t)b * M + i;
    tr[o] = phi[gi];
    ti[o] = phi[plane + gi];
    ur[o] = dphi[gi];
    ui[o] = dphi[plane + gi];
  }
  __syncthreads();
  for (int m = 1; m <= order; ++m) {
    const double inv = 1.0 / (double)m;
    for (int o = tid; o < NM; o += blockDim.x) {
      const int i = o / N, b = o % N;
      double sr = 0, si = 0, dr = 0, di = 0;
      packed_row_mac(ar, ai, M, i, tr, ti, N, b, sr, si);    // A T
      packed_row_mac(dar, dai, M, i, tr, ti, N, b, dr, di);  // dA T
      packed_row_mac(ar, ai, M, i, ur, ui, N, b, dr, di);    // + A dT
      nr[o] = sr * inv;
      ni[o] = si * inv;
      vr[o] = dr * inv;
      vi[o] = di * inv;
    }
    __syncthreads();
    for (int o = tid; o < NM; o += blockDim.x) {
      const int i = o / N, b = o % N;
      const int64_t gi = base + (int64_t)b * M + i;
      // accumulate into global (this walker's columns belong to this CTA only)
      phi[gi] += nr[o];
      phi[plane + gi] += ni[o];
      dphi[gi] += vr[o];
      dphi[plane + gi] += vi[o];
    }
    double* t0 = tr; tr = nr; nr = t0;
    double* t1 = ti; ti = ni; ni = t1;
    double* t2 = ur; ur = vr; vr = t2;
    double* t3 = ui; ui = vi; vi = t3;
    __syncthreads();
  }
}

// ---- overlap / Gauss-Jordan / Theta / weight update with tangents (FP64) ----
struct OvTanArgs {
  const double *src, *dsrc;       // propagated Phi', dPhi' (update mode)
  double *phi, *dphi, *theta, *dtheta;
  const double* psi;
  double *logO, *dlogO, *w, *dlogw;
  int* alive;
  const double *aux, *daux;
  int* flags;
  int M, N, n_up, Nw, mode;
  double log_shift, dlog_shift;
};

__global__ void __launch_bounds__(kT) k_overlap_tan(OvTanArgs a) {
  extern __shared__ double sm[];
  const int wk = blockIdx.x, tid = threadIdx.x, M = a.M, N = a.N;
  const int nmax = max(a.n_up, N - a.n_up);
  double* ph = sm;                        // [2][nmax][M]
  double* dp = ph + 2 * nmax * M;         // [2][nmax][M]
  double* th = dp + 2 * nmax * M;         // [2][nmax][M]
  double* aug = th + 2 * nmax * M;        // [2][nmax][2 nmax]
  double* dO = aug + 4 * nmax * nmax;     // [2][nmax][nmax]
  double* fac = dO + 2 * nmax * nmax;     // [2 + 2 nmax]
  __shared__ double s_ld[2], s_dld[2];
  __shared__ int s_piv, s_bad;
  const bool live = a.alive[wk] != 0;
  const bool upd = (a.mode == OV_UPDATE) && live;
  const double* src = upd ? a.src : a.phi;
  const double* dsrc = upd ? a.dsrc : a.dphi;
  const int64_t plane = (int64_t)a.Nw * N * M, wbase = (int64_t)wk * N * M;
  if (tid == 0) { s_ld[0] = s_ld[1] = s_dld[0] = s_dld[1] = 0.0; s_bad = 0; }
  for (int sp = 0; sp < 2; ++sp) {
    const int n0 = sp == 0 ? 0 : a.n_up, ns = sp == 0 ? a.n_up : N - a.n_up;
    if (ns == 0) continue;
    const int w2 = 2 * ns;
    __syncthreads();
    for (int e = tid; e < ns * M; e += blockDim.x) {
      const int64_t gi = wbase + (int64_t)n0 * M + e;
      ph[e] = src[gi];
      ph[nmax * M + e] = src[plane + gi];
      dp[e] = dsrc[gi];
      dp[nmax * M + e] = dsrc[plane + gi];
    }
    __syncthreads();
    for (int e = tid; e < ns * w2; e += blockDim.x) {
      const int r = e / w2, c = e % w2;
      double re = 0, im = 0;
      if (c < ns) {
        const double* pr = a.psi + (int64_t)(n0 + r) * M;
        double dre = 0, dim = 0;
        for (int i = 0; i < M; ++i) {
          const double p = __ldg(pr + i);
          re = fma(p, ph[c * M + i], re);
          im = fma(p, ph[nmax * M + c * M + i], im);
          dre = fma(p, dp[c * M + i], dre);
          dim = fma(p, dp[nmax * M + c * M + i], dim);
        }
        dO[r * ns + c] = dre;
        dO[ns * ns + r * ns + c] = dim;
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
    const bool bad = s_bad != 0;
    // dlog O_s = tr(O^{-1} dO) = sum_ab Oinv[a][b] dO[b][a]
    if (!bad && tid < 32) {
      double sr = 0, si = 0;
      for (int e = tid; e < ns * ns; e += 32) {
        const int aa = e / ns, bb = e % ns;
        const cplx v = cmul({ar[aa * w2 + ns + bb], ai[aa * w2 + ns + bb]},
                            {dO[bb * ns + aa], dO[ns * ns + bb * ns + aa]});
        sr += v.re;
        si += v.im;
      }
      for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_down_sync(0xffffffffu, sr, o);
        si += __shfl_down_sync(0xffffffffu, si, o);
      }
      if (tid == 0) { s_dld[0] += sr; s_dld[1] += si; }
    }
    // pass 1: Theta = Phi Oinv (shared + global); the propagated dPhi goes to the state
    for (int e = tid; e < ns * M; e += blockDim.x) {
      const int b = e / M, i = e % M;
      double re = 0, im = 0;
      if (!bad)
        for (int c = 0; c < ns; ++c) {
          const double orr = ar[c * w2 + ns + b], oi = ai[c * w2 + ns + b];
          const double xr = ph[c * M + i], xi = ph[nmax * M + c * M + i];
          re = fma(xr, orr, fma(-xi, oi, re));
          im = fma(xr, oi, fma(xi, orr, im));
        }
      th[b * M + i] = re;
      th[nmax * M + b * M + i] = im;
      const int64_t gi = wbase + (int64_t)(n0 + b) * M + i;
      a.theta[gi] = re;
      a.theta[plane + gi] = im;
      if (upd) {
        a.phi[gi] = ph[b * M + i];
        a.phi[plane + gi] = ph[nmax * M + b * M + i];
        a.dphi[gi] = dp[b * M + i];
        a.dphi[plane + gi] = dp[nmax * M + b * M + i];
      }
    }
    __syncthreads();
    // pass 2: Y = dPhi - Theta dO, in place of dPhi (entry (c, i) needs only its own dPhi)
    for (int e = tid; e < ns * M; e += blockDim.x) {
      const int c = e / M, i = e % M;
      double yr = dp[c * M + i], yi = dp[nmax * M + c * M + i];
      for (int d = 0; d < ns; ++d) {
        const double tr_ = th[d * M + i], ti_ = th[nmax * M + d * M + i];
        const double dr_ = dO[d * ns + c], di_ = dO[ns * ns + d * ns + c];
        yr -= tr_ * dr_ - ti_ * di_;
        yi -= tr_ * di_ + ti_ * dr_;
      }
      dp[c * M + i] = yr;
      dp[nmax * M + c * M + i] = yi;
    }
    __syncthreads();
    // pass 3: dTheta = Y Oinv
    for (int e = tid; e < ns * M; e += blockDim.x) {
      const int b = e / M, i = e % M;
      double dre = 0, dim = 0;
      if (!bad)
        for (int c = 0; c < ns; ++c) {
          const double orr = ar[c * w2 + ns + b], oi = ai[c * w2 + ns + b];
          const double yr = dp[c * M + i], yi = dp[nmax * M + c * M + i];
          dre = fma(yr, orr, fma(-yi, oi, dre));
          dim = fma(yr, oi, fma(yi, orr, dim));
        }
      const int64_t gi = wbase + (int64_t)(n0 + b) * M + i;
      a.dtheta[gi] = dre;
      a.dtheta[plane + gi] = dim;
    }
  }
  __syncthreads();
  if (tid != 0) return;
  const bool bad = s_bad != 0;
  const double ld_re = s_ld[0], ld_im = s_ld[1], dld_re = s_dld[0], dld_im = s_dld[1];
  if (bad || !isfinite(ld_re) || !isfinite(ld_im)) {
    atomicAdd(a.flags, 1);
    if (upd || a.mode == OV_REFRESH) {
      a.w[wk] = 0.0;
      a.w[a.Nw + wk] = 0.0;
      a.alive[wk] = 0;
      a.dlogw[wk] = 0.0;
    }
    return;
  }
  if (!upd) {
    a.logO[wk] = ld_re;
    a.logO[a.Nw + wk] = ld_im;
    a.dlogO[wk] = dld_re;
    a.dlogO[a.Nw + wk] = dld_im;
    return;
  }
  const double* x = a.aux + 4 * (int64_t)wk;
  const double* dx = a.daux + 4 * (int64_t)wk;
  const double lr_re = x[0] + ld_re - a.logO[wk];
  const double lr_im = x[1] + ld_im - a.logO[a.Nw + wk];
  const double li_re = lr_re + x[2] + a.log_shift;
  const double dlr_re = dx[0] + dld_re - a.dlogO[wk];
  const double dlr_im = dx[1] + dld_im - a.dlogO[a.Nw + wk];
  const double dli_re = dlr_re + dx[2] + a.dlog_shift;
  a.logO[wk] = ld_re;
  a.logO[a.Nw + wk] = ld_im;
  a.dlogO[wk] = dld_re;
  a.dlogO[a.Nw + wk] = dld_im;
  const double cs = cos(lr_im);
  const double nw = a.w[wk] * exp(li_re) * fmax(0.0, cs);
  if (nw > 0.0) {
    a.w[wk] = nw;
    a.dlogw[wk] += dli_re - tan(lr_im) * dlr_im;
  } else {
    a.w[wk] = 0.0;
    a.alive[wk] = 0;
    a.dlogw[wk] = 0.0;
  }
  a.w[a.Nw + wk] = 0.0;
}

// ---- MGS with the same column operations on dPhi ----
__global__ void __launch_bounds__(128) k_mgs_tan(double* __restrict__ phi, double* __restrict__ dphi,
                                                 const int* __restrict__ alive, int M, int N,
                                                 int n_up, int Nw) {
  extern __shared__ double sm[];
  const int wk = blockIdx.x, tid = threadIdx.x;
  if (!alive[wk]) return;
  const int NM = N * M;
  double* vr = sm;
  double* vi = vr + NM;
  double* ur = vi + NM;
  double* ui = ur + NM;
  double* red = ui + NM;
  const int64_t plane = (int64_t)Nw * NM, base = (int64_t)wk * NM;
  for (int e = tid; e < NM; e += blockDim.x) {
    vr[e] = phi[base + e];
    vi[e] = phi[plane + base + e];
    ur[e] = dphi[base + e];
    ui[e] = dphi[plane + base + e];
  }
  __syncthreads();
  for (int sp = 0; sp < 2; ++sp) {
    const int n0 = sp == 0 ? 0 : n_up, n1 = sp == 0 ? n_up : N;
    for (int j = n0; j < n1; ++j) {
      double* xr = vr + j * M;
      double* xi = vi + j * M;
      double* yr = ur + j * M;
      double* yi = ui + j * M;
      for (int q = n0; q < j; ++q) {
        const double* qr = vr + q * M;
        const double* qi = vi + q * M;
        const double* zr = ur + q * M;
        const double* zi = ui + q * M;
        double s[2] = {0, 0};
        for (int i = tid; i < M; i += blockDim.x) {
          s[0] += qr[i] * xr[i] + qi[i] * xi[i];
          s[1] += qr[i] * xi[i] - qi[i] * xr[i];
        }
        block_allsum<2>(s, red);
        for (int i = tid; i < M; i += blockDim.x) {
          xr[i] -= s[0] * qr[i] - s[1] * qi[i];
          xi[i] -= s[0] * qi[i] + s[1] * qr[i];
          yr[i] -= s[0] * zr[i] - s[1] * zi[i];
          yi[i] -= s[0] * zi[i] + s[1] * zr[i];
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
        yr[i] *= inv;
        yi[i] *= inv;
      }
      __syncthreads();
    }
  }
  for (int e = tid; e < NM; e += blockDim.x) {
    phi[base + e] = vr[e];
    phi[plane + base + e] = vi[e];
    dphi[base + e] = ur[e];
    dphi[plane + base + e] = ui[e];
  }
}

// ---- local energy and its tangent (FP64) ----
constexpr int G_CH = 4;
__global__ void __launch_bounds__(kT) k_energy_tan(const double* __restrict__ theta,
                                                   const double* __restrict__ dtheta,
                                                   const double* __restrict__ Ltil,
                                                   const double* __restrict__ htil,
                                                   const double* __restrict__ htilP,
                                                   double* __restrict__ eloc,
                                                   double* __restrict__ deloc, int M, int N,
                                                   int n_up, int X, int Nw) {
  extern __shared__ double sm[];
  const int wk = blockIdx.x, tid = threadIdx.x, NM = N * M;
  const int nu = n_up, nd = N - n_up, nn = nu * nu + nd * nd;
  double* thr = sm;
  double* thi = thr + NM;
  double* dhr = thi + NM;
  double* dhi = dhr + NM;
  double* Tr = dhi + NM;          // [G_CH][nn]
  double* Ti = Tr + G_CH * nn;
  double* Ur = Ti + G_CH * nn;    // dT
  double* Ui = Ur + G_CH * nn;
  double* red = Ui + G_CH * nn;
  const int64_t plane = (int64_t)Nw * NM, base = (int64_t)wk * NM;
  double acc[4] = {0, 0, 0, 0};   // E (re, im), dE (re, im)
  for (int e = tid; e < NM; e += blockDim.x) {
    const int n = e / M, i = e % M;
    const double vr = theta[base + e], vi = theta[plane + base + e];
    const double wr = dtheta[base + e], wi = dtheta[plane + base + e];
    thr[i * N + n] = vr;
    thi[i * N + n] = vi;
    dhr[i * N + n] = wr;
    dhi[i * N + n] = wi;
    const double h = __ldg(htil + e), hp = __ldg(htilP + e);
    acc[0] = fma(h, vr, acc[0]);
    acc[1] = fma(h, vi, acc[1]);
    acc[2] += hp * vr + h * wr;
    acc[3] += hp * vi + h * wi;
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
      double sr = 0, si = 0, ur = 0, ui = 0;
      for (int i = 0; i < M; ++i) {
        const double l = __ldg(lrow + i);
        sr = fma(l, thr[i * N + n0 + b], sr);
        si = fma(l, thi[i * N + n0 + b], si);
        ur = fma(l, dhr[i * N + n0 + b], ur);
        ui = fma(l, dhi[i * N + n0 + b], ui);
      }
      Tr[e] = sr;
      Ti[e] = si;
      Ur[e] = ur;
      Ui[e] = ui;
    }
    __syncthreads();
    for (int e = tid; e < gc * nn; e += blockDim.x) {
      const int gl = e / nn, r = e % nn;
      int et;
      if (r < nu * nu) { const int a = r / nu, b = r % nu; et = b * nu + a; }
      else { const int r2 = r - nu * nu; const int a = r2 / nd, b = r2 % nd; et = nu * nu + b * nd + a; }
      const cplx t = {Tr[e], Ti[e]}, tt = {Tr[gl * nn + et], Ti[gl * nn + et]};
      const cplx dtt = {Ur[gl * nn + et], Ui[gl * nn + et]};
      const cplx p = cmul(t, tt), dpv = cmul(t, dtt);
      acc[0] -= 0.5 * p.re;
      acc[1] -= 0.5 * p.im;
      acc[2] -= dpv.re;   // d(1/2 sum T_ab T_ba) = sum T_ab dT_ba
      acc[3] -= dpv.im;
    }
    for (int gl = tid; gl < gc; gl += blockDim.x) {
      double cr = 0, ci = 0, dr = 0, di = 0;
      for (int a = 0; a < nu; ++a) {
        cr += Tr[gl * nn + a * nu + a]; ci += Ti[gl * nn + a * nu + a];
        dr += Ur[gl * nn + a * nu + a]; di += Ui[gl * nn + a * nu + a];
      }
      for (int a = 0; a < nd; ++a) {
        const int q = gl * nn + nu * nu + a * nd + a;
        cr += Tr[q]; ci += Ti[q]; dr += Ur[q]; di += Ui[q];
      }
      acc[0] += 0.5 * (cr * cr - ci * ci);
      acc[1] += cr * ci;
      acc[2] += cr * dr - ci * di;   // d(1/2 rho^2) = rho drho
      acc[3] += cr * di + ci * dr;
    }
    __syncthreads();
  }
  block_sum<4>(acc, red);
  if (tid == 0) {
    eloc[wk] = acc[0];
    eloc[Nw + wk] = acc[1];
    deloc[wk] = acc[2];
    deloc[Nw + wk] = acc[3];
  }
}

// per repeat: sum w Re E_L, sum w, sum (dw Re E_L + w Re dE_L), sum dw   (dw = w dlog w)
__global__ void __launch_bounds__(256) k_mixed_sum_tan(const double* __restrict__ w,
                                                       const double* __restrict__ dlogw,
                                                       const double* __restrict__ eloc,
                                                       const double* __restrict__ deloc,
                                                       double* out, int Nw, int R) {
  __shared__ double red[4 * 8 + 4];
  const int r = blockIdx.x;
  const int64_t k0 = ((int64_t)r * Nw + R - 1) / R, k1 = ((int64_t)(r + 1) * Nw + R - 1) / R;
  double acc[4] = {0, 0, 0, 0};
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const double wk = w[k];
    if (wk == 0.0) continue;   // dead: contributes nothing (its E_L need not be finite)
    const double dw = wk * dlogw[k];
    acc[0] += wk * eloc[k];
    acc[1] += wk;
    acc[2] += dw * eloc[k] + wk * deloc[k];
    acc[3] += dw;
  }
  block_sum<4>(acc, red);
  if (threadIdx.x == 0)
    for (int q = 0; q < 4; ++q) out[4 * r + q] = acc[q];
}

size_t smem_overlap_tan(const Ctx& c) {
  const size_t nmax = c.n_up > c.N - c.n_up ? c.n_up : c.N - c.n_up;
  return sizeof(double) * (6 * nmax * c.M + 4 * nmax * nmax + 2 * nmax * nmax + 2 * nmax + 2);
}
size_t smem_taylor_tan(const Ctx& c) { return sizeof(double) * 8 * (size_t)c.N * c.M; }
size_t smem_mgs_tan(const Ctx& c) { return sizeof(double) * (4 * (size_t)c.N * c.M + 64); }
size_t smem_energy_tan(const Ctx& c) {
  const size_t nu = c.n_up, nd = c.N - c.n_up, nn = nu * nu + nd * nd;
  return sizeof(double) * (4 * (size_t)c.N * c.M + 4 * G_CH * nn + 64);
}

}  // namespace

bool tangent_fits(const Ctx& c) {
  return smem_taylor_tan(c) <= 200 * 1024 && smem_energy_tan(c) <= 200 * 1024 &&
         smem_mgs_tan(c) <= 200 * 1024 && smem_overlap_tan(c) <= 200 * 1024;
}

cudaError_t prepare_tangent_kernels(const Ctx& c) {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_overlap_tan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_overlap_tan(c))) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_taylor_tan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_taylor_tan(c))) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_mgs_tan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_mgs_tan(c))) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_energy_tan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_energy_tan(c));
}

cudaError_t launch_fields_tan(const Ctx& c, const double* fields, cudaStream_t s) {
  FieldTanArgs a;
  a.rhobar = c.rhobar; a.drhobar = c.drhobar; a.rho_mf = c.rho_mf; a.fields = fields;
  a.U = c.U; a.dU = c.dU; a.aux = c.aux; a.daux = c.daux; a.step = c.d_step;
  a.key = make_uint2((uint32_t)(c.opt.seed & 0xffffffffull), (uint32_t)(c.opt.seed >> 32));
  a.k0 = (uint32_t)c.opt.walker_offset;
  a.X = c.X; a.Nw = c.Nw; a.sqrt_dt = c.sqrt_dt; a.fb_cap = c.opt.fb_cap;
  k_fields_tan<<<c.Nw, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_taylor_tan(const Ctx& c, cudaStream_t s) {
  k_taylor_tan<<<c.Nw, kT, smem_taylor_tan(c), s>>>(c.phi2, c.dphi2, c.Avhs, c.dAvhs, c.M, c.N,
                                                    c.Nw, c.P, c.opt.taylor_order);
  return cudaGetLastError();
}

cudaError_t launch_overlap_tan(const Ctx& c, int mode, cudaStream_t s) {
  OvTanArgs a;
  a.src = c.theta; a.dsrc = c.dtheta;  // Phi', dPhi' are staged in the Theta buffers
  a.phi = c.phi; a.dphi = c.dphi; a.theta = c.theta; a.dtheta = c.dtheta;
  a.psi = c.psi; a.logO = c.logO; a.dlogO = c.dlogO; a.w = c.w; a.dlogw = c.dlogw;
  a.alive = c.alive; a.aux = c.aux; a.daux = c.daux; a.flags = c.d_flags;
  a.M = c.M; a.N = c.N; a.n_up = c.n_up; a.Nw = c.Nw; a.mode = mode;
  a.log_shift = -c.opt.dt * (c.c_mf - c.e_trial);
  a.dlog_shift = c.opt.dt * c.de_trial;
  k_overlap_tan<<<c.Nw, kT, smem_overlap_tan(c), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_mgs_tan(const Ctx& c, cudaStream_t s) {
  k_mgs_tan<<<c.Nw, 128, smem_mgs_tan(c), s>>>(c.phi, c.dphi, c.alive, c.M, c.N, c.n_up, c.Nw);
  return cudaGetLastError();
}

cudaError_t launch_energy_tan(const Ctx& c, cudaStream_t s) {
  k_energy_tan<<<c.Nw, kT, smem_energy_tan(c), s>>>(c.theta, c.dtheta, c.Ltil, c.htil, c.htilP,
                                                    c.eloc, c.deloc, c.M, c.N, c.n_up, c.X, c.Nw);
  return cudaGetLastError();
}

cudaError_t launch_mixed_sum_tan(const Ctx& c, double* out, cudaStream_t s) {
  k_mixed_sum_tan<<<c.R, 256, 0, s>>>(c.w, c.dlogw, c.eloc, c.deloc, out, c.Nw, c.R);
  return cudaGetLastError();
}

}  // namespace afq
