"""Pins of the oracle's Algorithm P (Sec. 2, steps 1-4) and its compaction in
candidate order: the exact lattice acceptance count against pi/4, observed
acceptance against the binomial law, brute-force accept bits on small inputs,
the closed forms of step 4, uniformity of s (Sec. 2), and normality."""
import math

import numpy as np
import pytest

import oracle
from stats import check_standard_normal_moments, ks_critical, ks_distance, normal_cdf

KEY = 0x5EED0001
H = 1 << 23


def test_lattice_accept_count_is_pi_over_4():
    a = oracle.lattice_accept_count()
    # Gauss circle problem: |A - pi R^2| is far below the perimeter 2 pi R for R = 2^23.
    assert abs(a - math.pi * 2.0 ** 46) < 2 * math.pi * H
    # the count is even in each coordinate sign pattern except the axes: sanity of range
    assert 0.78 * 2 ** 48 < a < 0.79 * 2 ** 48


@pytest.mark.parametrize("half_width", [1, 2, 3, 4, 5, 7, 8, 16, 31, 100, 181, 1024, 3000])
def test_lattice_accept_count_equals_enumeration(half_width):
    # exact pin of the count: every lattice point of half-width H enumerated,
    # with the strict bound s < 1 (a^2 + b^2 = H^2 rejected, e.g. (-H, 0)) and
    # the origin rejected (s = 0), as step 3 and the S = 0 reading fix them
    a = np.arange(-half_width, half_width, dtype=np.int64)
    s = a[:, None] * a[:, None] + a[None, :] * a[None, :]
    want = int(np.count_nonzero((s > 0) & (s < half_width * half_width)))
    assert oracle.lattice_accept_count(half_width) == want


def test_lattice_accept_count_small_cases_by_hand():
    # H = 1: only (-1,-1), (-1,0), (0,-1), (0,0); none has 0 < s < 1.
    # H = 2: the eight neighbours of the origin with |a|,|b| <= 1 (s = 1 or 2 < 4);
    # (-2, 0) and (0, -2) sit on the circle s = 4 and are rejected.
    assert oracle.lattice_accept_count(1) == 0
    assert oracle.lattice_accept_count(2) == 8


def test_accept_bits_brute_force():
    ncand = 4096
    acc, kx, ky = oracle.polar_candidates(ncand, KEY, 5)
    w = oracle.philox_blocks(ncand // 2, KEY, 5).astype(np.int64)
    ex = (w[:, [0, 2]] >> 8).ravel() - H      # candidate 2b uses words 0,1; 2b+1 words 2,3
    ey = (w[:, [1, 3]] >> 8).ravel() - H
    np.testing.assert_array_equal(kx, ex)
    np.testing.assert_array_equal(ky, ey)
    s_int = [int(a) * int(a) + int(b) * int(b) for a, b in zip(ex, ey)]
    want = np.array([1 if 0 < s < (1 << 46) else 0 for s in s_int], dtype=np.uint8)
    np.testing.assert_array_equal(acc, want)


def test_acceptance_rate_binomial():
    ncand = 1 << 22
    acc, _, _ = oracle.polar_candidates(ncand, KEY, 0)
    p = oracle.lattice_accept_count() / 2.0 ** 48
    k = int(acc.sum())
    assert abs(k - ncand * p) < 5 * math.sqrt(ncand * p * (1 - p))
    # uniforms per normal: 2 uniforms per candidate, 2 normals per accepted pair -> 4/pi
    assert abs(ncand / k - 4 / math.pi) < 2e-3


def test_stream_is_compaction_in_candidate_order():
    n = 2001
    mu, sigma = -0.5, 1.75
    out, cand, nxt, ncand = oracle.polar(n, mu, sigma, KEY, 3)
    acc, kx, ky = oracle.polar_candidates(ncand, KEY, 3)
    accepted = np.nonzero(acc)[0]
    assert accepted.size == (n + 1) // 2
    np.testing.assert_array_equal(cand, accepted)
    assert acc[ncand - 1] == 1                       # stops at the last needed pair
    pts = oracle.polar_points(kx[accepted], ky[accepted], mu, sigma).ravel()
    np.testing.assert_array_equal(out, pts[:n])      # odd n drops the last y
    assert nxt == 3 + cand[-1] // 2 + 1
    out2, cand2, _, _ = oracle.polar(n + 1, mu, sigma, KEY, 3)
    np.testing.assert_array_equal(out2[:n], out)
    np.testing.assert_array_equal(oracle.polar_at(cand[:7], mu, sigma, KEY, 3).ravel(), out[:14])


def test_step4_closed_forms():
    n = 1 << 16
    out, cand, _, ncand = oracle.polar(n, 0.0, 1.0, KEY, 0)
    acc, kx, ky = oracle.polar_candidates(ncand, KEY, 0)
    z = out.reshape(-1, 2)
    a = kx[cand].astype(np.float64)
    b = ky[cand].astype(np.float64)
    s = (a * a + b * b) * 2.0 ** -46
    # exp(-(zx^2 + zy^2)/2) = s: the radius of step 4 inverts to s
    np.testing.assert_allclose(np.exp(-(z[:, 0] ** 2 + z[:, 1] ** 2) / 2), s, rtol=1e-12)
    # the direction of (zx, zy) is that of (x, y): same signs, cross product zero
    assert np.all(np.sign(z[:, 0]) == np.sign(a)) and np.all(np.sign(z[:, 1]) == np.sign(b))
    np.testing.assert_allclose(z[:, 0] * b - z[:, 1] * a, 0.0, atol=1e-9 * H)
    # s of accepted pairs is uniform on [0, 1) (Sec. 2)
    assert ks_distance(s, lambda t: np.clip(t, 0, 1)) < ks_critical(s.size)


def test_special_lattice_points():
    kx = np.array([-H, 0, 1, 0, -1, H - 1, 3, H - 1], dtype=np.int32)
    ky = np.array([0, 0, 0, -1, 0, 4096, 4, 0], dtype=np.int32)
    out = oracle.polar_points(kx, ky, 0.0, 1.0)
    np.testing.assert_array_equal(oracle.polar_accept_points(kx, ky), [0, 0, 1, 1, 1, 0, 1, 1])
    assert np.all(np.isnan(out[0]))     # S = 2^46: s = 1 is rejected (s >= 1)
    assert np.all(np.isnan(out[1]))     # S = 0: rejected (division by s)
    zmax = math.sqrt(2 * 46 * math.log(2.0))   # smallest s = 2^-46: the tail bound
    np.testing.assert_allclose(out[2], [zmax, 0.0], rtol=1e-14)
    np.testing.assert_allclose(out[3], [0.0, -zmax], rtol=1e-14)
    np.testing.assert_allclose(out[4], [-zmax, 0.0], rtol=1e-14)
    assert np.all(np.isnan(out[5]))     # (2^23-1)^2 + 2^24 = 2^46 + 1: rejected
    # S = 25: s = 25 * 2^-46, r^2 = -2 ln s, (zx, zy) = r (3, 4) / 5
    r = math.sqrt(-2 * math.log(25 * 2.0 ** -46))
    np.testing.assert_allclose(out[6], [0.6 * r, 0.8 * r], rtol=1e-14)
    # S = (2^23-1)^2 just below 2^46: s -> 1, z -> 0 like sqrt(2(1 - s))
    d = 1.0 - (H - 1) ** 2 * 2.0 ** -46
    np.testing.assert_allclose(out[7, 0], math.sqrt(-2 * math.log1p(-d)) / math.sqrt(1 - d)
                               * (H - 1) / H, rtol=1e-9)
    assert out[7, 1] == 0.0


def test_normality():
    n = 1_000_000
    out, _, _, _ = oracle.polar(n, 0.0, 1.0, KEY, 0)
    check_standard_normal_moments(out)
    assert ks_distance(out, normal_cdf) < ks_critical(n)
    x, y = out.reshape(-1, 2).T
    assert abs(float(np.mean(x * y))) < 5.0 / math.sqrt(n / 2)


def test_mu_sigma_affine_and_tiny_n():
    z, _, _, _ = oracle.polar(1000, 0.0, 1.0, KEY, 0)
    x, _, _, _ = oracle.polar(1000, 1.5, 0.25, KEY, 0)
    np.testing.assert_allclose(x, 1.5 + 0.25 * z, atol=1e-14)
    o1, c1, n1, _ = oracle.polar(1, 0.0, 1.0, KEY, 0)
    assert o1.size == 1 and c1.size == 1 and n1 == c1[0] // 2 + 1
    o0, c0, n0, k0 = oracle.polar(0, 0.0, 1.0, KEY, 42)
    assert o0.size == 0 and n0 == 42 and k0 == 0
