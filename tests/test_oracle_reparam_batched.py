"""Pins of the oracle's reparameterised sample (x = mu + sigma z, z from B1)
against FP64 central finite differences of the loss sum(w x^2), and of the
batched oracle against the single-stream oracles it is made of."""
import numpy as np
import pytest

import oracle
from paper_1004_3105_gb300 import workloads

KEY = workloads.KEY_REPARAM


def _loss(mu, sigma, w, n, inner):
    x = oracle.reparam_fwd(mu, sigma, n, inner, KEY, 0)
    return float(np.sum(w.astype(np.float64) * x * x)), x


@pytest.mark.parametrize("shape,pshape,inner", [
    ((16, 24), (16, 24), 1),     # elementwise
    ((16, 24), (1,), 1),         # scalar mu, sigma: full reduction
    ((16, 24), (24,), 1),        # trailing-axis broadcast
    ((16, 24), (16, 1), 24),     # leading-axis broadcast
])
def test_gradient_matches_central_differences(shape, pshape, inner):
    rng = np.random.Generator(np.random.PCG64(5))
    n = int(np.prod(shape))
    mu = rng.standard_normal(size=pshape).astype(np.float32).ravel()
    sigma = rng.uniform(0.1, 2.0, size=pshape).astype(np.float32).ravel()
    w = rng.uniform(-1, 1, size=n).astype(np.float32)
    _, x = _loss(mu, sigma, w, n, inner)
    g = (2.0 * w.astype(np.float64) * x).astype(np.float32)
    dmu, dsig = oracle.reparam_bwd(g, mu.size, inner, KEY, 0)
    # The loss is quadratic in each parameter, so a central difference is exact
    # up to rounding; the step is taken on float32 parameters and the realised
    # step (an exact difference of two floats) is what we divide by.
    for p in range(mu.size):
        for arr, grad in ((mu, dmu), (sigma, dsig)):
            h = np.float32(2.0 ** -8)
            hi, lo = arr.copy(), arr.copy()
            hi[p] = arr[p] + h
            lo[p] = arr[p] - h
            step = float(hi[p]) - float(lo[p])
            lp, _ = _loss(hi if arr is mu else mu, hi if arr is sigma else sigma, w, n, inner)
            lm, _ = _loss(lo if arr is mu else mu, lo if arr is sigma else sigma, w, n, inner)
            fd = (lp - lm) / step
            # g was rounded to float32 before the backward: allow for that
            assert abs(fd - grad[p]) <= 1e-6 * (1.0 + abs(fd)) + 1e-7 * np.sum(np.abs(g)), (p, fd, grad[p])


def test_reparam_z_is_b1_stream():
    n = 1000
    mu = np.zeros(n, dtype=np.float32)
    sigma = np.ones(n, dtype=np.float32)
    np.testing.assert_array_equal(oracle.reparam_fwd(mu, sigma, n, 1, KEY, 3),
                                  oracle.boxmuller(n, 0.0, 1.0, KEY, 3))


def test_batched_is_single_streams():
    wl = workloads.batched_workload(k=12, len_lo=1, len_hi=3000)
    out = oracle.batched(wl.total, wl.as_dict())
    for j in range(12):
        o, n = int(wl.offset[j]), int(wl.n[j])
        mu, sg = float(wl.mu[j]), float(wl.sigma[j])
        if wl.method[j] == 0:
            want = oracle.boxmuller(n, mu, sg, int(wl.key[j]), 0)
        else:
            want = oracle.polar(n, mu, sg, int(wl.key[j]), 0)[0]
        np.testing.assert_array_equal(out[o:o + n], want)
    assert not np.any(np.isnan(out))
