"""The oracle's point evaluators (b3_points, p2_points, ratio_points), which
the GPU point tests check the kernels against at hand-picked inputs.  Pinned
here to (1) the oracle's own streams, fed the same words, and (2) for
Algorithm R's accept test (Sec. 5, step 3), to 50-digit arithmetic at the
lattice points next to the boundary, where a wrong term or rounding in the
double-precision decision would show first."""
import math

import numpy as np
import pytest

import oracle
from lattice_points import M23, M24, ratio_boundary, ratio_relative_gap, u24

KEY = 0x5EED0003
MU, SIGMA = 0.75, 1.25


def test_b3_points_reproduce_stream():
    npairs = 5000
    ref = oracle.b3(2 * npairs, MU, SIGMA, KEY, 3)
    w = oracle.philox_blocks((3 * npairs + 3) // 4, KEY, 3).ravel()[:3 * npairs].reshape(-1, 3)
    got = oracle.b3_points(u24(w[:, 0]), u24(w[:, 1]), u24(w[:, 2]), MU, SIGMA)
    np.testing.assert_array_equal(got.ravel(), ref)


def test_p2_points_reproduce_stream():
    n = 10000
    out, cand, _, _ = oracle.polar_p2(n, MU, SIGMA, KEY, 3)
    _, kx, ky = oracle.polar_candidates(int(cand[-1]) + 1, KEY, 3)
    np.testing.assert_array_equal(oracle.p2_points(kx[cand], ky[cand], MU, SIGMA).ravel(), out)


def test_ratio_points_reproduce_stream():
    n = 10000
    out, cand, _, nc = oracle.ratio(n, MU, SIGMA, KEY, 3)
    w = oracle.philox_blocks((nc + 1) // 2, KEY, 3)
    u = u24(w[:, [0, 2]].ravel())[:nc]
    v = u24(w[:, [1, 3]].ravel())[:nc]
    acc, vals = oracle.ratio_points(u, v, MU, SIGMA)
    np.testing.assert_array_equal(acc, oracle.ratio_candidates(nc, KEY, 3))
    np.testing.assert_array_equal(vals[cand], out)


def test_ratio_boundary_decisions_match_exact_arithmetic():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    k, j = ratio_boundary()
    acc, _ = oracle.ratio_points(k * 2.0 ** -24, j * 2.0 ** -24, 0.0, 1.0)
    e = mp.e
    exact = np.array([2 * mp.mpf(int(jj) - M23) ** 2 <= e * mp.mpf(M24 - int(kk)) ** 2 * -mp.log1p(-mp.mpf(int(kk)) / M24)
                      for kk, jj in zip(k, j)])
    np.testing.assert_array_equal(acc.astype(bool), exact)
    gap = ratio_relative_gap(k, j)
    # the set reaches the boundary closely: most points sit within the float
    # screen's margin, and a few at the widest point (u = 1 - e^-1/2,
    # a = -2^23) within 1e-12, where only the double decision can tell
    assert (gap < 1e-5).sum() > 20000
    near = gap < 1e-12
    assert near.sum() >= 5 and np.all(j[near] == 0)
    # u = 0 (b = 2^24, L = 0) accepts a = 0 alone
    z = k == 0
    np.testing.assert_array_equal(acc[z].astype(bool), j[z] == M23)


def test_ratio_region_is_widest_at_one_minus_exp_minus_half():
    # The boundary |v - 1/2| = (1 - u) sqrt(-e ln(1 - u) / 2) peaks at
    # 1 - u = e^-1/2, where it is exactly 1/2: the region just fits the unit
    # square, so the lattice edge a = -2^23 (v = 0) is never accepted.
    k, j = ratio_boundary()
    acc, _ = oracle.ratio_points(k * 2.0 ** -24, j * 2.0 ** -24, 0.0, 1.0)
    assert not acc[j == 0].any()
    t = math.exp(-0.5)
    assert abs(t * math.sqrt(-math.e * math.log(t) / 2) - 0.5) < 1e-15
