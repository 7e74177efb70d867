"""Pins of the oracle's Method B3 (Sec. 3), Method P2 (Sec. 4, step 4a) and
Algorithm R (Sec. 5) to facts other than the oracle itself: inverse relations
against the uniform stream, the uniformity claims the paper makes, the
acceptance rate the paper states, an equivalent form of the accept test, and
normality."""
import math

import numpy as np

import oracle
from stats import check_standard_normal_moments, ks_critical, ks_distance, normal_cdf

KEY = 0x5EED0001


def words(nwords, key, counter):
    return oracle.philox_blocks((nwords + 3) // 4, key, counter).ravel()[:nwords]


# ----------------------------------------------------------------------- B3
def test_b3_radius_and_angle_invert_to_uniforms():
    n = 1 << 14
    mu, sigma = 0.5, 1.5
    out = oracle.b3(n, mu, sigma, KEY, 3).reshape(-1, 2) - mu
    w = words(3 * (n // 2), KEY, 3).reshape(-1, 3)
    u = (w >> 8).astype(np.float64) * 2.0 ** -24
    m = np.maximum(u[:, 0], u[:, 1])
    # step 5 returns c r sqrt2 then s r sqrt2: (x^2 + y^2) / (2 sigma^2) = -ln(1 - m^2)
    rr = (out[:, 0] ** 2 + out[:, 1] ** 2) / (2 * sigma ** 2)
    np.testing.assert_allclose(np.exp(-rr), 1.0 - m * m, rtol=1e-12, atol=1e-15)
    # angle: atan2(s, c) = 2 pi u3 - pi
    ok = np.hypot(out[:, 0], out[:, 1]) > 1e-6
    ang = np.arctan2(out[ok, 1], out[ok, 0])
    d = (ang - (2 * np.pi * u[ok, 2] - np.pi)) / (2 * np.pi)
    assert np.max(np.abs(d - np.round(d))) < 1e-12


def test_b3_max_squared_is_uniform():
    # step 2: u = max(u1, u2)^2 is uniform on [0, 1) (Sec. 3)
    w = words(3 * 200000, KEY, 0).reshape(-1, 3)
    u = (w[:, :2] >> 8).astype(np.float64) * 2.0 ** -24
    m2 = np.max(u, axis=1) ** 2
    assert ks_distance(m2, lambda t: np.clip(t, 0, 1)) < ks_critical(m2.size)


def test_b3_normality():
    n = 1_000_000
    z = oracle.b3(n, 0.0, 1.0, KEY, 0)
    check_standard_normal_moments(z)
    assert ks_distance(z, normal_cdf) < ks_critical(n)
    x, y = z.reshape(-1, 2).T
    assert abs(float(np.mean(x * y))) < 5.0 / math.sqrt(n / 2)


# ----------------------------------------------------------------------- P2
def test_p2_same_candidates_as_p_and_radius_uses_one_minus_s():
    n = 20001
    mu, sigma = -1.0, 0.5
    out, cand, nxt, _ = oracle.polar_p2(n, mu, sigma, KEY, 11)
    _, pcand, pnxt, _ = oracle.polar(n, mu, sigma, KEY, 11)
    np.testing.assert_array_equal(cand, pcand)      # steps 1-3 are Algorithm P's
    assert nxt == pnxt
    acc, kx, ky = oracle.polar_candidates(int(cand[-1]) + 1, KEY, 11)
    a = kx[cand].astype(np.float64)
    b = ky[cand].astype(np.float64)
    s = (a * a + b * b) * 2.0 ** -46
    z = (np.concatenate([out, [np.nan]]) if n % 2 else out).reshape(-1, 2) - mu
    z = z[:-1] if n % 2 else z
    m = z.shape[0]
    # step 4a: (zx^2 + zy^2) / (2 sigma^2) = -ln(1 - s): the radius comes from 1 - s, not s
    np.testing.assert_allclose(np.exp(-(z[:, 0] ** 2 + z[:, 1] ** 2) / (2 * sigma ** 2)), 1.0 - s[:m], rtol=1e-11)
    assert np.all(np.sign(z[:, 0]) == np.sign(a[:m]))


def test_p2_normality():
    n = 1_000_000
    out, _, _, _ = oracle.polar_p2(n, 0.0, 1.0, KEY, 0)
    check_standard_normal_moments(out)
    assert ks_distance(out, normal_cdf) < ks_critical(n)


# ------------------------------------------------------------------------ R
def test_ratio_acceptance_rate_is_papers():
    # Sec. 5: 8 / sqrt(pi e) ~ 2.74 uniforms per normal, two per candidate, so
    # the acceptance probability is sqrt(pi e) / 4 ~ 0.7306
    ncand = 1 << 22
    acc = oracle.ratio_candidates(ncand, KEY, 0)
    p = math.sqrt(math.pi * math.e) / 4
    k = int(acc.sum())
    assert abs(k - ncand * p) < 5 * math.sqrt(ncand * p * (1 - p))
    assert abs(2 * ncand / k - 8 / math.sqrt(math.pi * math.e)) < 5e-3


def test_ratio_accept_bits_match_multiplied_out_form():
    # x^2 <= -4 ln(1-u) with x = sqrt(8/e)(v - 1/2)/(1 - u) is, multiplied by
    # (1 - u)^2, 2 (v - 1/2)^2 <= -e (1 - u)^2 ln(1 - u)
    ncand = 1 << 16
    acc = oracle.ratio_candidates(ncand, KEY, 7)
    w = oracle.philox_blocks(ncand // 2, KEY, 7).astype(np.int64)
    u = ((w[:, [0, 2]] >> 8).ravel()).astype(np.float64) * 2.0 ** -24
    v = ((w[:, [1, 3]] >> 8).ravel()).astype(np.float64) * 2.0 ** -24
    want = (2 * (v - 0.5) ** 2 <= -math.e * (1 - u) ** 2 * np.log1p(-u)).astype(np.uint8)
    np.testing.assert_array_equal(acc, want)


def test_ratio_stream_and_normality():
    n = 1_000_000
    out, cand, nxt, nc = oracle.ratio(n, 0.0, 1.0, KEY, 0)
    check_standard_normal_moments(out)
    assert ks_distance(out, normal_cdf) < ks_critical(n)
    acc = oracle.ratio_candidates(nc, KEY, 0)
    np.testing.assert_array_equal(np.flatnonzero(acc), cand)
    assert nxt == cand[-1] // 2 + 1
    np.testing.assert_array_equal(oracle.ratio_at(cand[:50], 0.0, 1.0, KEY, 0), out[:50])
