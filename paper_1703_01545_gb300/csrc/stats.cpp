// Host statistics of the correlated-sampling protocol (Sec. II.B, Fig. 1) and the
// Flyvbjerg-Petersen reblocking error.  Plain C++, usable without a GPU.
#include <cmath>
#include <vector>

#include "../../include/afqmc.h"

namespace {
// mean and standard error sd/sqrt(R) (sample sd) of v[0..R)
void mean_se(const double* v, int R, double& mean, double& se) {
  double s = 0;
  for (int i = 0; i < R; ++i) s += v[i];
  mean = s / R;
  if (R < 2) { se = NAN; return; }
  double q = 0;
  for (int i = 0; i < R; ++i) q += (v[i] - mean) * (v[i] - mean);
  se = std::sqrt(q / (R - 1)) / std::sqrt((double)R);
}
}  // namespace

extern "C" afqmc_status afqmc_delta_E_stats(const double* dE, const double* taus, int n_meas, int R,
                                            double tau_eq, double* mean_tau, double* se_tau,
                                            double* est) {
  if (!dE || !taus || n_meas < 0 || R < 1) return AFQMC_ERR_ARG;
  for (int m = 0; m < n_meas; ++m) {
    double mu, se;
    mean_se(dE + (size_t)m * R, R, mu, se);
    if (mean_tau) mean_tau[m] = mu;
    if (se_tau) se_tau[m] = se;
  }
  if (!est) return AFQMC_OK;
  est[0] = est[1] = est[2] = NAN;
  int m0 = -1;
  for (int m = 0; m < n_meas; ++m)
    if (taus[m] >= tau_eq) { m0 = m; break; }
  if (m0 < 0) return AFQMC_OK;
  std::vector<double> run(R, 0.0), c(R);
  double best_se = INFINITY, best_mu = NAN, best_tau = NAN, last_mu = NAN;
  bool any = false;
  for (int m = m0; m < n_meas; ++m) {
    const double cnt = (double)(m - m0 + 1);
    for (int r = 0; r < R; ++r) {
      run[r] += dE[(size_t)m * R + r];
      c[r] = run[r] / cnt;
    }
    double mu, se;
    mean_se(c.data(), R, mu, se);
    last_mu = mu;
    if (!std::isnan(se) && se < best_se) {
      best_se = se;
      best_mu = mu;
      best_tau = taus[m];
      any = true;
    }
  }
  if (any) {
    est[0] = best_mu;
    est[1] = best_se;
    est[2] = best_tau;
  } else {
    est[0] = last_mu;
    est[1] = NAN;
    est[2] = taus[n_meas - 1];
  }
  return AFQMC_OK;
}

extern "C" double afqmc_reblock_error(const double* series, int n) {
  if (!series || n < 1) return NAN;
  std::vector<double> x(series, series + n);
  double best = 0;
  while ((int)x.size() >= 16) {
    const size_t k = x.size();
    double mu = 0;
    for (double v : x) mu += v;
    mu /= (double)k;
    double var = 0;
    for (double v : x) var += (v - mu) * (v - mu);
    var /= (double)k;
    best = std::fmax(best, std::sqrt(var / (double)(k - 1)));
    std::vector<double> y(k / 2);
    for (size_t i = 0; i < k / 2; ++i) y[i] = 0.5 * (x[2 * i] + x[2 * i + 1]);
    x.swap(y);
  }
  return best;
}
