"""Pins of the oracle's counter-based field stream (Philox-4x32-10 + Box-Muller)."""
import numpy as np

from golden_util import philox_kat
from oracle.philox import box_muller, gaussian_fields, philox4x32_10, uniforms53


def test_philox_known_answers():
    for ctr, key, want in philox_kat():
        got = philox4x32_10(np.array(ctr, np.uint32), np.array(key, np.uint32))
        assert [int(v) for v in got] == want


def test_uniform_extremes_and_box_muller_closed_form():
    # all-ones words -> u1 = 1 exactly (r = 0), u2 = 1 - 2^-53
    w = np.array([[0xFFFFFFFF] * 4], dtype=np.uint32)
    u1, u2 = uniforms53(w)
    assert u1[0] == 1.0 and u2[0] == 1.0 - 2.0 ** -53
    # all-zero words -> u1 = 2^-53 (never 0), u2 = 0
    u1, u2 = uniforms53(np.zeros((1, 4), np.uint32))
    assert u1[0] == 2.0 ** -53 and u2[0] == 0.0
    z0, z1 = box_muller(np.array([np.exp(-0.5)]), np.array([0.125]))
    assert np.isclose(z0[0], np.cos(np.pi / 4)) and np.isclose(z1[0], np.sin(np.pi / 4))


def test_normal_moments():
    x = gaussian_fields(12345, 3, np.arange(2000), 100).ravel()
    n = x.size
    assert abs(x.mean()) < 5 / np.sqrt(n)
    assert abs(x.var() - 1) < 5 * np.sqrt(2 / n)
    kurt = np.mean(x ** 4) / x.var() ** 2
    assert abs(kurt - 3) < 5 * np.sqrt(24 / n)


def test_fields_shared_across_systems_and_distinct_across_walkers_steps():
    a = gaussian_fields(99, 7, np.arange(5), 31)
    b = gaussian_fields(99, 7, np.arange(5), 24)
    np.testing.assert_array_equal(a[:, :24], b)          # truncation keeps x_g (config 4)
    c = gaussian_fields(99, 7, np.array([3]), 31)
    np.testing.assert_array_equal(a[3:4], c)             # depends on (seed, t, k, g) only
    d = gaussian_fields(99, 8, np.arange(5), 31)
    e = gaussian_fields(100, 7, np.arange(5), 31)
    assert not np.any(a == d) and not np.any(a == e)
    assert not np.any(a[0] == a[1])
