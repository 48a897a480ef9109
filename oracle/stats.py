"""Repeat statistics of the correlated-sampling protocol (Sec. II.B, Fig. 1).

* Per imaginary-time point: mean of the energy difference over the N_r repeats
  and its standard error, sd / sqrt(N_r) (sample sd, ddof = 1).
* Cumulative averages: for each repeat, the running mean of the measurements
  taken at tau >= tau_eq up to each tau.
* Final value: mean and SE of the cumulative averages over repeats at the tau
  where that SE is smallest (the earliest one when several are equal).
* Reblocking (Flyvbjerg and Petersen 1989, cited in Sec. II.B): repeatedly
  average neighbour pairs; the error estimate of block level l is
  sqrt(var_l / (n_l - 1)); the plateau (largest value among levels with at
  least 16 blocks) is returned.
"""
import numpy as np


def per_tau(dE):
    """dE [n_meas, R] -> (mean [n_meas], se [n_meas])."""
    dE = np.asarray(dE, dtype=np.float64)
    R = dE.shape[1]
    mean = dE.mean(axis=1)
    se = dE.std(axis=1, ddof=1) / np.sqrt(R) if R > 1 else np.full(dE.shape[0], np.nan)
    return mean, se


def cumulative(dE, taus, tau_eq):
    """Running averages [n_meas - m0, R] over measurements with tau >= tau_eq; returns (taus, C)."""
    dE = np.asarray(dE, dtype=np.float64)
    taus = np.asarray(taus, dtype=np.float64)
    sel = taus >= tau_eq
    if not np.any(sel):
        return taus[:0], dE[:0]
    m0 = int(np.argmax(sel))
    d = dE[m0:]
    C = np.cumsum(d, axis=0) / np.arange(1, d.shape[0] + 1)[:, None]
    return taus[m0:], C


def delta_e_estimate(dE, taus, tau_eq):
    """(mean, se, tau_at_min_se) of the cumulative averages at the earliest minimum SE."""
    t, C = cumulative(dE, taus, tau_eq)
    if C.shape[0] == 0:
        return np.nan, np.nan, np.nan
    mean, se = per_tau(C)
    if np.all(np.isnan(se)):
        return float(mean[-1]), float("nan"), float(t[-1])
    i = int(np.nanargmin(se))
    return float(mean[i]), float(se[i]), float(t[i])


def reblock(series, min_blocks: int = 16):
    """Flyvbjerg-Petersen error of the mean of an autocorrelated series."""
    x = np.asarray(series, dtype=np.float64)
    best = 0.0
    while x.size >= min_blocks:
        n = x.size
        err = np.sqrt(np.var(x, ddof=0) / (n - 1))
        best = max(best, err)
        n2 = n // 2
        x = 0.5 * (x[0:2 * n2:2] + x[1:2 * n2:2])
    return best
