"""The seeded input generators (paper_1004_3105_gb300/workloads.py) follow
the recipe the design states: 4096 streams with lengths log-uniform in
[10^2, 10^6], mu ~ U(-2, 2), sigma ~ U(0.1, 3), key = stream id, counter 0,
methods B1/Polar alternating, starts rounded up to the alignment; the
reparameterised inputs mu ~ N(0, 1), sigma ~ U(0.1, 2), w ~ U(-1, 1).  The
figures the design quotes for the bench's workload follow from them."""
import numpy as np
from scipy import stats

from paper_1004_3105_gb300 import workloads as W


def test_batched_recipe():
    wl = W.batched_workload(methods="mixed", align=4)
    again = W.batched_workload(methods="mixed", align=4)
    for f in ("offset", "n", "mu", "sigma", "key", "counter", "method"):
        np.testing.assert_array_equal(getattr(wl, f), getattr(again, f))   # seeded
    k = W.BATCH_STREAMS
    assert k == 4096 and wl.n.size == k
    assert wl.n.min() >= 100 and wl.n.max() <= 10 ** 6
    # log10(n) is uniform on [2, 6] (rounding n to integers moves it by < 0.005)
    assert stats.kstest((np.log10(wl.n) - 2.0) / 4.0, "uniform").pvalue > 1e-3
    # (float32 rounding can reach the upper end of a half-open range)
    assert np.all((wl.mu >= -2) & (wl.mu <= 2)) and np.all((wl.sigma >= 0.1) & (wl.sigma <= 3))
    np.testing.assert_array_equal(wl.key, np.arange(k, dtype=np.uint64))
    assert np.all(wl.counter == 0)
    np.testing.assert_array_equal(wl.method, np.arange(k) % 2)
    # packed back to back, each start rounded up to 4 elements (16 bytes of fp32)
    assert np.all(wl.offset % 4 == 0) and wl.offset[0] == 0
    assert np.all(wl.offset[1:] >= wl.offset[:-1] + wl.n[:-1])
    assert np.all(wl.offset[1:] - (wl.offset[:-1] + wl.n[:-1]) < 4)
    assert wl.total == wl.offset[-1] + wl.n[-1]
    # the figures quoted for the bench's workload
    assert wl.total == 443294224
    assert abs(np.mean(wl.n < 10 ** 4) - 0.5) < 0.03


def test_batched_method_mixes():
    b1 = W.batched_workload(methods="b1")
    p = W.batched_workload(methods="polar")
    assert np.all(b1.method == 0) and np.all(p.method == 1)
    np.testing.assert_array_equal(b1.n, p.n)   # same lengths, only the method differs
    dense = W.batched_workload(methods="mixed")
    np.testing.assert_array_equal(dense.offset[1:], np.cumsum(dense.n)[:-1])


def test_reparam_recipe():
    rw = W.reparam_workload()
    assert rw.mu.shape == rw.sigma.shape == rw.w.shape == W.REPARAM_SHAPE
    assert rw.mu.dtype == np.float32
    assert abs(float(rw.mu.mean())) < 5e-3 and abs(float(rw.mu.std()) - 1.0) < 5e-3
    assert np.all((rw.sigma >= 0.1) & (rw.sigma <= 2)) and np.all((rw.w >= -1) & (rw.w <= 1))


def test_sample_indices():
    idx = W.sample_indices(10 ** 6, 1000)
    assert idx[0] == 0 and idx[-1] == 10 ** 6 - 1
    assert np.all(np.diff(idx) > 0) and idx.size >= 1000
    np.testing.assert_array_equal(W.sample_indices(5, 100), np.arange(5))
