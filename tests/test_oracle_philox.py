"""Pins of the oracle's Philox4x32-10 and uniform map to sources other than itself:
the published known-answer vectors and cuRAND's host Philox4x32-10 generator."""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_known_answer_vectors():
    rows = _kat_rows()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = oracle.philox4x32_10(ctr, key)
        assert [int(x) for x in got] == want


def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if path:
            try:
                return ctypes.CDLL(path)
            except OSError:
                pass
    return None


def _curand_host_philox(seed: int, nwords: int, offset: int = 0) -> np.ndarray:
    lib = _curand()
    if lib is None:
        pytest.skip("cuRAND host library not available")
    g = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    assert lib.curandCreateGeneratorHost(ctypes.byref(g), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(g, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(nwords, dtype=np.uint32)
        assert lib.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(nwords)) == 0
        return out
    finally:
        lib.curandDestroyGenerator(g)


# cuRAND's host generator runs 65536 interleaved subsequences: word block
# 65536*j + t of its output is Philox(ctr = (j, 0, t, 0), key = seed).  That
# layout was established empirically; it is cuRAND's, not ours.
CURAND_THREADS = 65536


@pytest.mark.parametrize("seed", [0x5EED0001, 0x123456789ABCDEF0])
def test_matches_curand_host_philox(seed):
    jmax = 4
    words = _curand_host_philox(seed, 4 * CURAND_THREADS * jmax).reshape(jmax, CURAND_THREADS, 4)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    rng = np.random.Generator(np.random.PCG64(3))
    for j in range(jmax):
        for t in list(range(8)) + list(rng.integers(0, CURAND_THREADS, size=24)):
            got = oracle.philox4x32_10([j, 0, int(t), 0], key)
            assert np.array_equal(got, words[j, t]), (j, t)
    # Our stream layout: block b of (key, counter) is ctr = (lo(counter+b), hi(counter+b), 0, 0).
    ours = oracle.philox_blocks(jmax, seed, 0)
    assert np.array_equal(ours, words[:, 0, :])


def test_uniform_map_against_curand_words():
    seed = 0x5EED0001
    words = _curand_host_philox(seed, 4 * CURAND_THREADS * 2).reshape(2, CURAND_THREADS, 4)
    u = oracle.uniform(8, seed, 0).reshape(2, 4)
    # u = (w >> 8) * 2^-24 with w the cuRAND word of the same block.
    assert np.array_equal(u * 2.0 ** 24, (words[:, 0, :] >> 8).astype(np.float64))


def test_uniform_lattice_and_range():
    n = 1 << 20
    u = oracle.uniform(n, 0x5EED0001, 12345)
    k = u * 2.0 ** 24
    assert np.array_equal(k, np.floor(k))          # on the 24-bit lattice
    assert k.min() >= 0 and k.max() <= 2 ** 24 - 1   # in [0, 1): never 1
    # low byte of k is uniform (chi-square, 255 dof; 0.1% critical value ~ 330)
    h = np.bincount((k.astype(np.int64) & 255), minlength=256)
    e = n / 256.0
    chi2 = float(np.sum((h - e) ** 2 / e))
    assert chi2 < 330.0, chi2
    # each output is its own 24-bit draw: consecutive elements uncorrelated
    d = u - u.mean()
    rho = float(np.mean(d[1:] * d[:-1]) / np.mean(d * d))
    assert abs(rho) < 5.0 / np.sqrt(n)


def test_counter_offsets_concatenate():
    a = oracle.uniform(40, 7, 100)
    b = oracle.uniform(20, 7, 105)   # block 105 = element 20 of the first stream
    assert np.array_equal(a[20:], b)
    c = oracle.uniform(8, 7, (1 << 32) - 1)  # counter carries into the high word
    w = oracle.philox4x32_10([0xFFFFFFFF, 0, 0, 0], [7, 0])
    w2 = oracle.philox4x32_10([0, 1, 0, 0], [7, 0])
    assert np.array_equal(c * 2.0 ** 24, np.concatenate([w >> 8, w2 >> 8]).astype(np.float64))
