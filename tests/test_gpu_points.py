"""The per-pair transforms at hand-picked lattice points, through
nrng_eval_points, against the oracle: the special points of Algorithm B1
(u = 0, u = 1 - 2^-24, v on the quadrant angles) and of Algorithm P
(S = 1, S = 2, S just below and at 2^46, s -> 1, the origin), Method P2's and
B3's switch to the upper branch at 8/9, and the lattice points next to
Algorithm R's accept boundary, which a stream reaches too rarely to test.
Accept decisions bit-exact (for R, wherever the boundary is farther than
1e-12 relative); values within the mode's tolerance."""
import numpy as np
import pytest
import torch

import lattice_points as LP
import oracle
import paper_1004_3105_gb300 as nr
from gpu_helpers import assert_close

pytestmark = pytest.mark.gpu
MU, SIGMA = 0.75, 1.25


def b1_words():
    rng = np.random.Generator(np.random.PCG64(5))
    ks = [0, 1, 2, 255, 1 << 12, (1 << 23) - 1, 1 << 23, (1 << 24) - 2, (1 << 24) - 1]
    js = [0, 1, 1 << 22, (1 << 22) + 1, 1 << 23, (1 << 23) - 1, 3 << 22, (1 << 24) - 1]
    k = np.array([a for a in ks for _ in js], dtype=np.uint64)
    j = np.array([b for _ in ks for b in js], dtype=np.uint64)
    # random low bytes: the lattice uses only the top 24 bits of each word
    low = rng.integers(0, 256, size=(k.size, 2), dtype=np.uint64)
    wu = (k << np.uint64(8)) | low[:, 0]
    wv = (j << np.uint64(8)) | low[:, 1]
    rnd = rng.integers(0, 1 << 32, size=(4096, 2), dtype=np.uint64)
    w = np.concatenate([np.stack([wu, wv], axis=1), rnd]).astype(np.uint32)
    return w


@pytest.mark.parametrize("mode", ["accurate", "fast", "b2"])
def test_b1_special_points(mode):
    w = b1_words()
    got, acc = nr.nrng_eval_points(nr.B1, torch.from_numpy(w.view(np.int32)).cuda(), MU, SIGMA, mode)
    u = (w[:, 0] >> 8).astype(np.float64) * 2.0 ** -24
    v = (w[:, 1] >> 8).astype(np.float64) * 2.0 ** -24
    ref = oracle.b1_points(u, v, MU, SIGMA)
    assert bool((acc == 1).all())
    assert_close(got.reshape(-1), ref.reshape(-1), MU, SIGMA, "accurate" if mode == "accurate" else "fast",
                 f"B1 points {mode}")
    # u = 0 gives r = 0: both outputs are exactly mu
    z = got.cpu().numpy()[(w[:, 0] >> 8) == 0]
    assert np.all(z == np.float32(MU))


def test_b1_accurate_every_lattice_radius_and_angle():
    """The accurate B1 transform over its whole domain: every radius k (2^24
    values, at t = 0, where sin = 0 and cos = 1 exactly, so y = r) and every
    angle t (2^24 values, at u = 1 - e^-1/2, where r is near 1), against the
    oracle.  The radius takes the hardware log2 of the exact 1 - u above
    u = 2^-9 (its absolute error moves r most there: measured 7.9e-7)
    and a three-term series below it.  A coordinate's error from the radius is
    at most the radius error and |z| <= r, so the radius is held to half the
    accurate bound, 2e-6 max(1, r).  The angle comes from the 1024-entry table
    with quadratic angle addition (under 1e-7 absolute): x, y within 5e-7
    absolute at r ~ 1."""
    n = 1 << 24
    idx = np.arange(n, dtype=np.uint64)
    w = np.stack([(idx << np.uint64(8)).astype(np.uint32), np.zeros(n, np.uint32)], axis=1)
    got, _ = nr.nrng_eval_points(nr.B1, torch.from_numpy(w.view(np.int32)).cuda(), 0.0, 1.0, "accurate")
    g = got.cpu().numpy().astype(np.float64)
    u = idx.astype(np.float64) * 2.0 ** -24
    ref = oracle.b1_points(u, np.zeros(n), 0.0, 1.0)
    assert np.all(g[:, 0] == 0.0)
    assert g[0, 1] == 0.0                                   # u = 0: r = 0
    rel = np.abs(g[1:, 1] - ref[1:, 1]) / np.maximum(1.0, ref[1:, 1])
    print(f"B1 accurate radius: max error {rel.max():.3e} max(1, r) at k = {int(np.argmax(rel)) + 1}")
    assert rel.max() <= 2e-6, f"radius: max error {rel.max():.3e} max(1, r) at k = {int(np.argmax(rel)) + 1}"
    k0 = int(LP.M24 * (1.0 - np.exp(-0.5)))
    w = np.stack([np.full(n, k0 << 8, np.uint32), (idx << np.uint64(8)).astype(np.uint32)], axis=1)
    got, _ = nr.nrng_eval_points(nr.B1, torch.from_numpy(w.view(np.int32)).cuda(), 0.0, 1.0, "accurate")
    g = got.cpu().numpy().astype(np.float64)
    ref = oracle.b1_points(np.full(n, k0 * 2.0 ** -24), u, 0.0, 1.0)
    err = np.abs(g - ref).max()
    assert err <= 5e-7, f"angle: max absolute error {err:.3e}"


def polar_points():
    m = 1 << 23
    pts = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, -1), (3, 4),
           (m - 1, 0), (0, m - 1), (-(m - 1), 0), (-m, 0), (0, -m), (-m, 1), (-m, -m),
           (m - 1, 1 << 11), (m - 1, (1 << 11) + 1), (m - 2, 4096), (5792, 5792)]
    rng = np.random.Generator(np.random.PCG64(6))
    # points just inside and just outside the unit circle (s -> 1)
    th = rng.uniform(0.0, 2.0 * np.pi, 2048)
    for eps in (0.0, 1e-7, 2e-6, -1e-7):
        r = (m - 1) * (1.0 - eps)
        pts += list(zip(np.clip(np.rint(r * np.cos(th)), -m, m - 1).astype(int),
                        np.clip(np.rint(r * np.sin(th)), -m, m - 1).astype(int)))
    # near the origin (s -> 0, the largest |z|) and uniform points
    pts += list(zip(rng.integers(-64, 65, 1024), rng.integers(-64, 65, 1024)))
    pts += list(zip(rng.integers(-m, m, 4096), rng.integers(-m, m, 4096)))
    return np.array(pts, dtype=np.int32)


def test_polar_accurate_radius():
    """ln s of the accurate Polar path at every S = k^2 (0 < k < 2^23, so s
    runs from 2^-46 to 1 - 2^-22) and at 4 M random lattice points: the
    radius |(x, y) - mu| = sigma sqrt(-2 ln s) against the oracle.  Below
    1 - s = 2^-8 the path takes a series in the exact complement; above it
    the hardware log2 of s (s rounded to 2^-23), whose error moves the radius
    most near 1 - s = 2^-8 (measured 9.3e-7) and less beyond.  A coordinate's
    error from the radius is at most the radius error and |z| <= r, so the
    radius is held to half the accurate bound, 2e-6 max(1, r)."""
    k = np.arange(1, 1 << 23, dtype=np.int64)
    rng = np.random.Generator(np.random.PCG64(21))
    rnd = rng.integers(-(1 << 23), 1 << 23, (1 << 22, 2))
    p = np.concatenate([np.stack([k, np.zeros_like(k)], axis=1), rnd]).astype(np.int32)
    S = p[:, 0].astype(np.int64) ** 2 + p[:, 1].astype(np.int64) ** 2
    p = p[(S > 0) & (S < (1 << 46))]
    got, acc = nr.nrng_eval_points(nr.POLAR, torch.from_numpy(p).cuda(), 0.0, 1.0, "accurate")
    assert bool((acc == 1).all())
    g = got.cpu().numpy().astype(np.float64)
    ref = oracle.polar_points(p[:, 0], p[:, 1], 0.0, 1.0)
    r_got, r_ref = np.hypot(g[:, 0], g[:, 1]), np.hypot(ref[:, 0], ref[:, 1])
    rel = np.abs(r_got - r_ref) / np.maximum(1.0, r_ref)
    print(f"Polar accurate radius: max error {rel.max():.3e} max(1, r) at {p[int(np.argmax(rel))]}")
    assert rel.max() <= 2e-6, f"max radius error {rel.max():.3e} max(1, r) at {p[int(np.argmax(rel))]}"


@pytest.mark.parametrize("mode", ["accurate", "fast"])
def test_polar_special_points(mode):
    p = polar_points()
    got, acc = nr.nrng_eval_points(nr.POLAR, torch.from_numpy(p).cuda(), MU, SIGMA, mode)
    want = oracle.polar_accept_points(p[:, 0], p[:, 1])
    acc = acc.cpu().numpy()
    assert np.array_equal(acc, want.astype(np.int32)), "accept decisions"
    # the boundary cases decide as Algorithm P's step 3 says
    S = p[:, 0].astype(np.int64) ** 2 + p[:, 1].astype(np.int64) ** 2
    assert np.array_equal(acc, ((S > 0) & (S < (1 << 46))).astype(np.int32))
    assert acc[0] == 0 and acc[11] == 0 and acc[13] == 0          # origin, S = 2^46, S > 2^46
    keep = np.flatnonzero(acc == 1)
    ref = oracle.polar_points(p[keep, 0], p[keep, 1], MU, SIGMA)
    assert_close(got[torch.from_numpy(keep).cuda()].reshape(-1), ref.reshape(-1), MU, SIGMA, mode,
                 f"Polar points {mode}")


def test_p2_special_points():
    p, S = LP.p2_points()
    pts = torch.from_numpy(p).cuda()
    got, acc = nr.nrng_eval_points(nr.POINTS_P2, pts, MU, SIGMA, "accurate")
    got_fast, _ = nr.nrng_eval_points(nr.POINTS_P2, pts, MU, SIGMA, "fast")
    # one mode: bit-identical values (NaN at rejected points, where they are meaningless)
    torch.testing.assert_close(got, got_fast, rtol=0, atol=0, equal_nan=True)
    acc = acc.cpu().numpy()
    assert np.array_equal(acc, ((S > 0) & (S < LP.S_ONE)).astype(np.int32)), "accept decisions"
    # both sides of the switch at 8/9 are reached closely, and s -> 1
    assert ((S > LP.S_SWITCH) & (S < LP.S_SWITCH + 10 ** 8)).sum() > 1000
    assert ((S <= LP.S_SWITCH) & (S > LP.S_SWITCH - 10 ** 8)).sum() > 1000
    assert ((S < LP.S_ONE) & (S > LP.S_ONE - 10 ** 9)).sum() > 1000
    keep = np.flatnonzero(acc == 1)
    ref = oracle.p2_points(p[keep, 0], p[keep, 1], MU, SIGMA)
    assert_close(got[torch.from_numpy(keep).cuda()].reshape(-1), ref.reshape(-1), MU, SIGMA, "fast", "P2 points")


@pytest.mark.parametrize("mode", ["accurate", "fast"])
def test_ratio_boundary_points(mode):
    w = LP.ratio_words()
    got, acc = nr.nrng_eval_points(nr.POINTS_RATIO, torch.from_numpy(w.view(np.int32)).cuda(), MU, SIGMA, mode)
    k = (w[:, 0] >> 8).astype(np.int64)
    j = (w[:, 1] >> 8).astype(np.int64)
    want, ref = oracle.ratio_points(k * 2.0 ** -24, j * 2.0 ** -24, MU, SIGMA)
    acc = acc.cpu().numpy()
    gap = LP.ratio_relative_gap(k, j)
    # most points lie inside the float screen's margin, so the double
    # decision takes them; within 1e-12 of the boundary (a handful of points
    # at the region's widest place) double rounding may decide either way
    assert (gap < 1e-5).sum() > 20000
    decided = gap >= 1e-12
    assert np.array_equal(acc[decided], want[decided].astype(np.int32)), "accept decisions"
    assert acc.sum() > 10000 and (acc == 0).sum() > 10000
    keep = np.flatnonzero((acc == 1) & (want == 1))
    assert_close(got[torch.from_numpy(keep).cuda(), 0], ref[keep], MU, SIGMA, mode, f"R points {mode}")
    assert bool((got[:, 1] == 0).all())


def test_b3_special_points():
    w = LP.b3_words()
    pts = torch.from_numpy(w.view(np.int32)).cuda()
    got, acc = nr.nrng_eval_points(nr.POINTS_B3, pts, MU, SIGMA, "accurate")
    got_fast, _ = nr.nrng_eval_points(nr.POINTS_B3, pts, MU, SIGMA, "fast")
    torch.testing.assert_close(got, got_fast, rtol=0, atol=0)   # one mode
    assert bool((acc == 1).all())
    ref = oracle.b3_points(LP.u24(w[:, 0]), LP.u24(w[:, 1]), LP.u24(w[:, 2]), MU, SIGMA)
    assert_close(got.reshape(-1), ref.reshape(-1), MU, SIGMA, "fast", "B3 points")
    m = np.maximum(w[:, 0] >> 8, w[:, 1] >> 8).astype(np.float64) * 2.0 ** -24
    assert (m * m > 8.0 / 9.0).sum() > 500 and ((m * m <= 8.0 / 9.0) & (m * m > 0.8888)).sum() > 500
    # u1 = u2 = 0 gives r = 0: both outputs are exactly mu
    z = m == 0
    assert z.any() and np.all(got.cpu().numpy()[z] == np.float32(MU))


def test_eval_points_validation():
    pts = torch.zeros((4, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(nr.NrngError):
        nr.nrng_eval_points(7, pts)
    with pytest.raises(nr.NrngError):
        nr.nrng_eval_points(5, pts)
    for kind in (nr.POLAR, nr.POINTS_P2, nr.POINTS_RATIO):
        with pytest.raises(nr.NrngError):
            nr.nrng_eval_points(kind, pts, mode="b2")
    with pytest.raises(ValueError):
        nr.nrng_eval_points(nr.POINTS_B3, pts)
    out, acc = nr.nrng_eval_points(nr.POLAR, pts[:0])
    assert out.shape == (0, 2) and acc.shape == (0,)
    out, acc = nr.nrng_eval_points(nr.POINTS_B3, torch.zeros((0, 3), dtype=torch.int32, device="cuda"))
    assert out.shape == (0, 2) and acc.shape == (0,)
