"""Hand-picked inputs for the point evaluators (nrng_eval_points and the
oracle's *_points functions): the places where a method changes branch or
decides on a boundary, which a Philox stream reaches too rarely to test.
Plain numpy; seeded."""
import math

import numpy as np

M23 = 1 << 23
M24 = 1 << 24
S_ONE = 1 << 46                                   # S = 2^46 is s = 1
S_SWITCH = int(8.0 / 9.0 * 70368744177664.0)      # P2/B3 switch to the upper branch at 8/9


def _words(top24, rng):
    """32-bit words with the given top 24 bits and random low bytes (the
    lattice maps use only the top 24 bits)."""
    top24 = np.asarray(top24, dtype=np.uint64)
    return ((top24 << np.uint64(8)) | rng.integers(0, 256, size=top24.shape, dtype=np.uint64)).astype(np.uint32)


def ratio_boundary(seed=11):
    """Lattice candidates (k, j) of Algorithm R on and next to the accept
    boundary 2 a^2 = e b^2 L (a = j - 2^23, b = 2^24 - k, L = -ln(1 - k 2^-24)):
    for each k, the integers a next to +-sqrt(e b^2 L / 2).  The k cover u = 0,
    the smallest u, the series range below u = 1/16 and the switch there, the
    widest point of the region (u = 1 - e^-1/2, where the boundary reaches
    a = -2^23), and u -> 1.  Returns (k, j) as int64 arrays."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ks = [0, 1, 2, 3, 7, 100, 4095, 4096, 4097]
    ks += list(range((1 << 20) - 4, (1 << 20) + 5))                      # u = 1/16
    widest = int(M24 * (1.0 - math.exp(-0.5)))
    ks += list(range(widest - 64, widest + 65))                         # the widest point
    ks += list(M24 - np.arange(1, 200))                                 # b = 1 .. 199
    ks += list(np.unique(np.exp(rng.uniform(0.0, math.log(1 << 20), 1500)).astype(np.int64)))
    ks += list(rng.integers(0, M24, 3000))
    k = np.unique(np.array(ks, dtype=np.int64))
    b = (M24 - k).astype(np.float64)
    A = np.sqrt(math.e * b * b * -np.log1p(-k * 2.0 ** -24) / 2.0)
    fa = np.floor(A).astype(np.int64)
    kk, aa = [], []
    for d in (-1, 0, 1, 2):
        for sgn in (1, -1):
            kk.append(k)
            aa.append(sgn * (fa + d))
    kk.append(k)
    aa.append(np.full(k.shape, -M23, dtype=np.int64))                  # the lattice edge
    k = np.concatenate(kk)
    a = np.concatenate(aa)
    keep = (a >= -M23) & (a < M23)
    ka = np.unique(np.stack([k[keep], a[keep] + M23], axis=1), axis=0)
    return ka[:, 0], ka[:, 1]


def ratio_words(seed=11):
    """ratio_boundary as Philox words, plus uniform random candidates."""
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    k, j = ratio_boundary(seed)
    wu = np.concatenate([_words(k, rng), rng.integers(0, 1 << 32, 4096, dtype=np.uint64).astype(np.uint32)])
    wv = np.concatenate([_words(j, rng), rng.integers(0, 1 << 32, 4096, dtype=np.uint64).astype(np.uint32)])
    return np.stack([wu, wv], axis=1)


def ratio_relative_gap(k, j):
    """|2 a^2 - e b^2 L| / (e b^2 L) in double precision (inf where L = 0)."""
    a = (np.asarray(j, dtype=np.int64) - M23).astype(np.float64)
    b = (M24 - np.asarray(k, dtype=np.int64)).astype(np.float64)
    rhs = math.e * b * b * -np.log1p(-np.asarray(k, dtype=np.float64) * 2.0 ** -24)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(rhs > 0, np.abs(2 * a * a - rhs) / rhs, np.inf)


def p2_points(seed=12):
    """Lattice points (kx', ky') for P2's step 4a: S on both sides of the
    switch at 8/9, s -> 1 (S up to 2^46 - 1), s -> 0, and uniform points."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = []
    th = rng.uniform(0.0, 2.0 * np.pi, 4096)
    for r in (math.sqrt(S_SWITCH) - 1.5, math.sqrt(S_SWITCH) - 0.5, math.sqrt(S_SWITCH), math.sqrt(S_SWITCH) + 0.5,
              math.sqrt(S_SWITCH) + 1.5):
        pts.append(np.stack([np.rint(r * np.cos(th)), np.rint(r * np.sin(th))], axis=1))
    for eps in (0.0, 1e-7, 2e-6, 1e-4):
        r = (M23 - 1) * (1.0 - eps)
        pts.append(np.stack([np.clip(np.rint(r * np.cos(th)), -M23, M23 - 1),
                             np.clip(np.rint(r * np.sin(th)), -M23, M23 - 1)], axis=1))
    pts.append(np.array([[M23 - 1, 0], [0, M23 - 1], [-(M23 - 1), 0], [M23 - 1, 1 << 11], [M23 - 2, 4096],
                         [1, 0], [0, -1], [1, 1], [3, 4], [-M23 + 1, 1]], dtype=np.float64))
    pts.append(rng.integers(-64, 65, (1024, 2)).astype(np.float64))
    pts.append(rng.integers(-M23, M23, (4096, 2)).astype(np.float64))
    p = np.concatenate(pts).astype(np.int32)
    S = p[:, 0].astype(np.int64) ** 2 + p[:, 1].astype(np.int64) ** 2
    return p, S


def b3_words(seed=13):
    """Word triples (w1, w2, w3) for B3: max(u1, u2)^2 on both sides of 8/9,
    the largest m (u -> 1), m = 0 and the smallest m, the quadrant angles and
    their neighbours, and uniform triples."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ksw = int(math.sqrt(8.0 / 9.0) * M24)
    ms = list(range(ksw - 40, ksw + 41)) + [M24 - 1, M24 - 2, M24 - 1000, 0, 1, 2, 1 << 12, 1 << 23]
    angles = []
    for q in (0, 1 << 22, 1 << 23, 3 << 22, M24 - 1):
        angles += [q, (q + 1) % M24, (q - 1) % M24]
    angles += list(rng.integers(0, M24, 8))
    m = np.array([a for a in ms for _ in angles], dtype=np.int64)
    t = np.array([b for _ in ms for b in angles], dtype=np.int64)
    other = (m * rng.uniform(0.0, 1.0, m.size)).astype(np.int64)      # the smaller of u1, u2
    first = rng.integers(0, 2, m.size).astype(bool)                    # which word holds the max
    k1 = np.where(first, m, other)
    k2 = np.where(first, other, m)
    w = np.stack([_words(k1, rng), _words(k2, rng), _words(t, rng)], axis=1)
    rnd = rng.integers(0, 1 << 32, (4096, 3), dtype=np.uint64).astype(np.uint32)
    eq = _words(np.repeat(rng.integers(0, M24, 64), 3).reshape(64, 3), rng)
    eq[:, 1] = eq[:, 0]                                                # u1 = u2
    return np.concatenate([w, rnd, eq])


def u24(w):
    """The lattice uniform k 2^-24 of a word (top 24 bits)."""
    return (np.asarray(w, dtype=np.uint32) >> np.uint32(8)).astype(np.float64) * 2.0 ** -24
