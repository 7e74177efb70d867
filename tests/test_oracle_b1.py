"""Pins of the oracle's Algorithm B1 (Sec. 2, steps 1-3, notes a and b):
the inverse relations between (x, y) and (u, v), hand-picked special cases,
the element layout against the uniform stream, and normality statistics."""
import math

import numpy as np

import oracle
from stats import check_standard_normal_moments, ks_critical, ks_distance, normal_cdf

KEY = 0x5EED0001


def test_radius_inverts_to_one_minus_u():
    # exp(-(x^2 + y^2) / (2 sigma^2)) = 1 - u, the inverse of step 2.
    n = 1 << 16
    sigma = 0.75
    z = oracle.boxmuller(n, 0.0, sigma, KEY, 0).reshape(-1, 2)
    u = oracle.uniform(n, KEY, 0).reshape(-1, 2)[:, 0]
    lhs = np.exp(-(z[:, 0] ** 2 + z[:, 1] ** 2) / (2 * sigma ** 2))
    np.testing.assert_allclose(lhs, 1.0 - u, rtol=1e-12, atol=1e-15)


def test_angle_is_two_pi_v():
    # atan2(x - mu, y - mu) recovers the angle 2 pi v modulo 2 pi.
    n = 1 << 16
    mu = 1.5
    z = oracle.boxmuller(n, mu, 1.0, KEY, 0).reshape(-1, 2) - mu
    v = oracle.uniform(n, KEY, 0).reshape(-1, 2)[:, 1]
    r = np.hypot(z[:, 0], z[:, 1])
    ok = r > 1e-6
    ang = np.arctan2(z[ok, 0], z[ok, 1]) / (2 * math.pi)      # in (-1/2, 1/2]
    d = (ang - v[ok]) - np.round(ang - v[ok])
    assert np.max(np.abs(d)) < 1e-12


def test_special_points():
    mu, sigma = 0.5, 2.0
    u = np.array([0.0, 0.5, 0.5, 0.5, 0.5, 1.0 - 2.0 ** -24])
    v = np.array([0.3, 0.0, 0.25, 0.5, 0.75, 0.125])
    out = oracle.b1_points(u, v, mu, sigma)
    r = sigma * math.sqrt(2.0 * math.log(2.0))   # u = 1/2: -2 ln(1/2) = 2 ln 2
    # u = 0: r = 0, both outputs equal mu
    assert out[0, 0] == mu and out[0, 1] == mu
    # v = 0: sin 0 = 0, cos 0 = 1
    np.testing.assert_allclose(out[1], [mu, mu + r], atol=1e-15)
    # v = 1/4: sin = 1, cos = 0
    np.testing.assert_allclose(out[2], [mu + r, mu], atol=1e-15)
    # v = 1/2: angle -pi (note b's interval), sin = 0, cos = -1
    np.testing.assert_allclose(out[3], [mu, mu - r], atol=1e-15)
    # v = 3/4: angle -pi/2, sin = -1, cos = 0
    np.testing.assert_allclose(out[4], [mu - r, mu], atol=1e-15)
    # largest u on the lattice: r = sigma sqrt(2 * 24 ln 2), the tail bound
    rmax = sigma * math.sqrt(48.0 * math.log(2.0))
    np.testing.assert_allclose(np.hypot(out[5, 0] - mu, out[5, 1] - mu), rmax, rtol=1e-14)
    np.testing.assert_allclose(out[5, 0] - mu, out[5, 1] - mu, rtol=1e-12)  # angle pi/4


def test_stream_layout_against_uniforms():
    # block b gives pairs (u, v) = (w0, w1) and (w2, w3); out[4b+2p] = x, out[4b+2p+1] = y
    n = 4096
    u = oracle.uniform(n, KEY, 77).reshape(-1, 2)
    pts = oracle.b1_points(u[:, 0], u[:, 1], -1.0, 3.0).ravel()
    np.testing.assert_array_equal(oracle.boxmuller(n, -1.0, 3.0, KEY, 77), pts)
    idx = np.array([0, 1, 2, 3, 1001, 4095])
    np.testing.assert_array_equal(oracle.boxmuller_at(idx, -1.0, 3.0, KEY, 77), pts[idx])


def test_normality():
    n = 1_000_000
    z = oracle.boxmuller(n, 0.0, 1.0, KEY, 0)
    check_standard_normal_moments(z)
    assert ks_distance(z, normal_cdf) < ks_critical(n)
    x, y = z.reshape(-1, 2).T
    rho = float(np.mean(x * y) - x.mean() * y.mean())
    assert abs(rho) < 5.0 / math.sqrt(n / 2)


def test_mu_sigma_affine():
    n = 1 << 14
    z = oracle.boxmuller(n, 0.0, 1.0, KEY, 9)
    x = oracle.boxmuller(n, 1.5, 0.25, KEY, 9)
    np.testing.assert_allclose(x, 1.5 + 0.25 * z, rtol=0, atol=1e-14)
