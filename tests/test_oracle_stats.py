"""Pins of the repeat statistics (Sec. II.B) and the reblocking estimate."""
import numpy as np

from oracle import stats


def test_per_tau_mean_and_standard_error():
    dE = np.array([[1.0, 2.0, 3.0, 6.0], [0.0, 0.0, 0.0, 0.0]])
    m, se = stats.per_tau(dE)
    assert m[0] == 3.0 and m[1] == 0.0
    assert np.isclose(se[0], np.sqrt(np.var([1, 2, 3, 6], ddof=1) / 4))
    assert se[1] == 0.0


def test_cumulative_and_earliest_minimum():
    taus = np.array([0.1, 0.2, 0.3, 0.4, 0.5])
    dE = np.array([[9, 9], [1, 3], [3, 1], [2, 2], [2, 2]], dtype=float)
    t, C = stats.cumulative(dE, taus, 0.2)
    np.testing.assert_allclose(t, [0.2, 0.3, 0.4, 0.5])
    np.testing.assert_allclose(C[:, 0], [1, 2, 2, 2])
    np.testing.assert_allclose(C[:, 1], [3, 2, 2, 2])
    mean, se, tmin = stats.delta_e_estimate(dE, taus, 0.2)
    assert mean == 2.0 and se == 0.0 and tmin == 0.3   # earliest of the equal minima


def test_reblocking_iid_and_ar1():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(2 ** 16)
    assert abs(stats.reblock(x) / (1 / np.sqrt(x.size)) - 1) < 0.25
    phi = 0.9
    y = np.empty(2 ** 17)
    y[0] = 0
    e = rng.standard_normal(y.size)
    for i in range(1, y.size):
        y[i] = phi * y[i - 1] + e[i]
    # AR(1): var = 1/(1-phi^2), integrated correlation factor (1+phi)/(1-phi)
    true = np.sqrt((1 / (1 - phi ** 2)) * (1 + phi) / (1 - phi) / y.size)
    assert abs(stats.reblock(y) / true - 1) < 0.3
