// Multi-determinant trial (Sec. II.D; the truncated CASSCF trials of Sec. III), FP64 path.
//
//   psi_T = sum_d c_d D_d, with real M x N determinants D_d.  For every walker and determinant
//   the single-determinant overlap kernel gives O_d = <D_d|phi> (as a log) and
//   Theta_d = Phi (D_d^T Phi)^{-1} (one grid row per determinant, no weight update).  Then,
//   per walker:
//     <psi_T|phi> = sum_d c_d O_d, formed relative to the largest |O_d|;
//     shares      w_d = c_d O_d / <psi_T|phi>;
//     force bias  rhobar_g = sum_d w_d rhobar_g,d  (rhobar_d the contraction of Eq. 9 with
//                 D_d's half-rotated Cholesky vectors; rhobar is linear in G = sum_d w_d G_d);
//     local energy E_L = sum_d w_d E_L,d  (<D_d|H|phi> = O_d E_L,d; the two-body part of E_L is
//                 not linear in G, so it is taken determinant by determinant);
//   and the weight update of Sec. II.A and II.D uses the ratio of <psi_T|phi>.
// A determinant with O_d = 0 (singular D_d^T Phi) contributes nothing: its Theta_d would need
// cofactor formulas, so walkers should start from a determinant outside the expansion.  The
// mean-field background <rho_g>_T, K and E_T are those of D_0 (the regular setup with D_0 as
// trial computes them).
#include <cmath>

#include "internal.h"

namespace afq {
namespace {

// Per walker: log <psi_T|phi> from the determinants' log overlaps, the shares w_d, and (update
// form, walkers alive on entry) the ratio, phase and weight update; a total overlap that is
// zero or not finite kills the walker and is counted.
__global__ void k_md_combine(const double* __restrict__ logOd, const double* __restrict__ coef,
                             int Nd, double* __restrict__ share, double* logO, double* w,
                             int* alive, const double* __restrict__ aux, int* flags, int Nw,
                             int update, int free_proj, double log_shift) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Nw) return;
  const bool upd = update && alive[k] != 0;
  if (update && !upd) return;                    // dead: frozen state, weight 0
  double top = -INFINITY;
  for (int d = 0; d < Nd; ++d) {
    const double r = logOd[(int64_t)d * 2 * Nw + k];
    if (coef[d] != 0.0 && isfinite(r) && r > top) top = r;
  }
  double sre = 0.0, sim = 0.0;
  if (isfinite(top))
    for (int d = 0; d < Nd; ++d) {
      const double r = logOd[(int64_t)d * 2 * Nw + k], i = logOd[(int64_t)d * 2 * Nw + Nw + k];
      if (coef[d] == 0.0 || !isfinite(r)) continue;
      double sn, cs;
      sincos(i, &sn, &cs);
      const double m = coef[d] * exp(r - top);
      sre += m * cs;
      sim += m * sn;
    }
  const double mag2 = sre * sre + sim * sim;
  const double lt_re = top + 0.5 * log(mag2), lt_im = atan2(sim, sre);
  const bool bad = !(mag2 > 0.0) || !isfinite(lt_re) || !isfinite(lt_im);
  for (int d = 0; d < Nd; ++d) {
    const double r = logOd[(int64_t)d * 2 * Nw + k], i = logOd[(int64_t)d * 2 * Nw + Nw + k];
    double sre_d = 0.0, sim_d = 0.0;
    if (!bad && coef[d] != 0.0 && isfinite(r)) {
      double sn, cs;
      sincos(i - lt_im, &sn, &cs);
      const double m = coef[d] * exp(r - lt_re);
      sre_d = m * cs;
      sim_d = m * sn;
    }
    share[(int64_t)d * 2 * Nw + k] = sre_d;
    share[(int64_t)d * 2 * Nw + Nw + k] = sim_d;
  }
  if (bad) {
    atomicAdd(flags, 1);
    w[k] = 0.0;
    w[Nw + k] = 0.0;
    alive[k] = 0;
    return;
  }
  if (!upd) {
    logO[k] = lt_re;
    logO[Nw + k] = lt_im;
    return;
  }
  const double* x = aux + 4 * (int64_t)k;
  const double lr_re = x[0] + lt_re - logO[k];
  const double lr_im = x[1] + lt_im - logO[Nw + k];
  const double li_re = lr_re + x[2] + log_shift;
  const double li_im = lr_im + x[3];
  logO[k] = lt_re;
  logO[Nw + k] = lt_im;
  if (free_proj) {
    const double mag = exp(li_re);
    double sn, cs;
    sincos(li_im, &sn, &cs);
    const double fr = mag * cs, fi = mag * sn, wr = w[k], wi = w[Nw + k];
    w[k] = wr * fr - wi * fi;
    w[Nw + k] = wr * fi + wi * fr;
  } else {
    const double nw = w[k] * exp(li_re) * fmax(0.0, cos(lr_im));
    if (nw > 0.0) {
      w[k] = nw;
    } else {
      w[k] = 0.0;
      alive[k] = 0;
    }
    w[Nw + k] = 0.0;
  }
}

// out[p][k][j] = sum_d share_d[k] part_d[p][k][j] (complex, planar [2][Nw][K] per determinant)
__global__ void k_md_mix(const double* __restrict__ share, const double* __restrict__ part,
                         double* __restrict__ out, int Nd, int Nw, int K) {
  const int64_t n = (int64_t)Nw * K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / K);
    double re = 0.0, im = 0.0;
    for (int d = 0; d < Nd; ++d) {
      const double sr = share[(int64_t)d * 2 * Nw + k], si = share[(int64_t)d * 2 * Nw + Nw + k];
      if (sr == 0.0 && si == 0.0) continue;
      const double* p = part + (int64_t)d * 2 * n;
      const double pr = p[e], pi = p[n + e];
      re += sr * pr - si * pi;
      im += sr * pi + si * pr;
    }
    out[e] = re;
    out[n + e] = im;
  }
}

// Phi <- Phi' for the walkers alive on entry to the weight update ([2][Nw][N][M])
__global__ void k_md_take_live(const double* __restrict__ src, double* __restrict__ phi,
                               const int* __restrict__ alive, int64_t NM, int Nw) {
  const int64_t n = 2 * (int64_t)Nw * NM;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)((e / NM) % Nw);
    if (alive[k]) phi[e] = src[e];
  }
}

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

}  // namespace

cudaError_t md_overlap(const Ctx& c, const double* src, int mode, cudaStream_t s) {
  const int64_t NM = (int64_t)c.N * c.M;
  const bool update = mode == OV_UPDATE;
  // the determinants' overlaps and Theta_d of Phi' (update) or of the current walkers
  cudaError_t e = launch_overlap_dets(c, update ? src : nullptr, s);
  if (e != cudaSuccess) return e;
  if (update) {
    k_md_take_live<<<grid_for(2 * c.Nw * NM), 256, 0, s>>>(src, c.phi, c.alive, NM, c.Nw);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_md_combine<<<(c.Nw + 127) / 128, 128, 0, s>>>(
      c.md_logO, c.md_coef, c.n_det, c.md_share, c.logO, c.w, c.alive, c.aux, c.d_flags, c.Nw,
      update ? 1 : 0, c.opt.mode == AFQMC_FREE, -c.opt.dt * (c.c_mf - c.e_trial));
  return cudaGetLastError();
}

cudaError_t md_force_bias(const Ctx& c, cudaStream_t s) {
  const int64_t NM = (int64_t)c.N * c.M;
  cudaError_t e = gemm_tn_f64(c.X, 2 * c.Nw, (int)NM, 1.0, c.md_Ltil, NM, (int64_t)c.X * NM,
                              c.md_theta, NM, 2 * (int64_t)c.Nw * NM, 0.0, c.md_rhobar, c.X,
                              2 * (int64_t)c.Nw * c.X, c.n_det, s, GEMM_FORCE_BIAS);
  if (e != cudaSuccess) return e;
  k_md_mix<<<grid_for((int64_t)c.Nw * c.X), 256, 0, s>>>(c.md_share, c.md_rhobar, c.rhobar,
                                                          c.n_det, c.Nw, c.X);
  return cudaGetLastError();
}

cudaError_t md_energy(const Ctx& c, cudaStream_t s) {
  const int64_t NM = (int64_t)c.N * c.M;
  for (int d = 0; d < c.n_det; ++d) {
    Ctx v = c;
    v.theta = c.md_theta + (int64_t)d * 2 * c.Nw * NM;
    v.Ltil = c.md_Ltil + (int64_t)d * c.X * NM;
    v.htil = c.md_htil + (int64_t)d * NM;
    v.eloc = c.md_eloc + (int64_t)d * 2 * c.Nw;
    cudaError_t e = launch_energy(v, s);
    if (e != cudaSuccess) return e;
  }
  k_md_mix<<<grid_for(c.Nw), 256, 0, s>>>(c.md_share, c.md_eloc, c.eloc, c.n_det, c.Nw, 1);
  return cudaGetLastError();
}

}  // namespace afq
