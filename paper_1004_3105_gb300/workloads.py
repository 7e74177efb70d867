"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds none of the generators' arithmetic: it only draws the
parameters a caller hands to a generator (keys, counters, stream lengths,
mu/sigma arrays, upstream gradients) from numpy's PCG64 with fixed seeds, so
that the CUDA path and the CPU oracle are fed identical inputs.  The normal
variates themselves are always drawn by the generator under test from its
(key, counter) pair.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# Keys and counters of the fixed workloads.
KEY_MAIN = 0x5EED0001        # B1/Polar single-stream runs and the precision sweep
KEY_REPARAM = 0x5EED0002     # z of the reparameterised sample
COUNTER0 = 0

# Workload sizes.
N_PARITY_B1 = 1 << 20        # B1, mu=0, sigma=1, accurate, fp32
N_PARITY_POLAR = 1 << 26     # Polar and B1 side by side
N_FULL = 1 << 28             # the headline single-stream size (1 GiB of fp32)
SWEEP_MU, SWEEP_SIGMA = 1.5, 0.25
REPARAM_SHAPE = (1024, 8192)
BATCH_STREAMS = 4096
BATCH_SEED = 7
BATCH_LEN_LO, BATCH_LEN_HI = 1e2, 1e6


@dataclass
class BatchedWorkload:
    """k independent streams packed back to back in one output buffer."""
    offset: np.ndarray   # int64 [k], element offset of each stream in the output
    n: np.ndarray        # int64 [k], normals in each stream
    mu: np.ndarray       # float32 [k]
    sigma: np.ndarray    # float32 [k]
    key: np.ndarray      # uint64 [k], the stream id
    counter: np.ndarray  # uint64 [k], 0
    method: np.ndarray   # int32 [k], 0 = B1, 1 = Polar
    total: int           # sum of n

    def as_dict(self):
        return {f: getattr(self, f) for f in
                ("offset", "n", "mu", "sigma", "key", "counter", "method")}


def batched_workload(k: int = BATCH_STREAMS, seed: int = BATCH_SEED, methods: str = "mixed",
                     len_lo: float = BATCH_LEN_LO, len_hi: float = BATCH_LEN_HI,
                     align: int = 1) -> BatchedWorkload:
    """Stream lengths log-uniform in [len_lo, len_hi], mu ~ U(-2, 2),
    sigma ~ U(0.1, 3), key = stream id, counter 0.

    methods: "b1" (all Box-Muller), "polar" (all Polar) or "mixed" (i mod 2).
    align: round every stream's start offset up to a multiple of this many
    elements (1 packs them densely, so most streams start unaligned).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    e = rng.uniform(np.log10(len_lo), np.log10(len_hi), size=k)
    n = np.rint(10.0 ** e).astype(np.int64)
    mu = rng.uniform(-2.0, 2.0, size=k).astype(np.float32)
    sigma = rng.uniform(0.1, 3.0, size=k).astype(np.float32)
    ids = np.arange(k, dtype=np.int64)
    if methods == "b1":
        method = np.zeros(k, dtype=np.int32)
    elif methods == "polar":
        method = np.ones(k, dtype=np.int32)
    elif methods == "mixed":
        method = (ids % 2).astype(np.int32)
    else:
        raise ValueError(f"unknown methods {methods!r}")
    offset = np.zeros(k, dtype=np.int64)
    pos = 0
    for j in range(k):
        pos = (pos + align - 1) // align * align
        offset[j] = pos
        pos += int(n[j])
    return BatchedWorkload(offset=offset, n=n, mu=mu, sigma=sigma,
                           key=ids.astype(np.uint64), counter=np.zeros(k, dtype=np.uint64),
                           method=method, total=int(pos))


@dataclass
class ReparamWorkload:
    mu: np.ndarray      # float32, N(0, 1)
    sigma: np.ndarray   # float32, U(0.1, 2)
    w: np.ndarray       # float32, U(-1, 1): loss = sum(w * x^2)


def reparam_workload(shape=REPARAM_SHAPE, seed: int = 0xC5) -> ReparamWorkload:
    rng = np.random.Generator(np.random.PCG64(seed))
    mu = rng.standard_normal(size=shape).astype(np.float32)
    sigma = rng.uniform(0.1, 2.0, size=shape).astype(np.float32)
    w = rng.uniform(-1.0, 1.0, size=shape).astype(np.float32)
    return ReparamWorkload(mu=mu, sigma=sigma, w=w)


def sample_indices(n: int, m: int, seed: int = 11) -> np.ndarray:
    """m sorted distinct indices in [0, n) that always include both ends."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = min(m, n)
    idx = rng.choice(n, size=m, replace=False) if m < n else np.arange(n)
    idx = np.unique(np.concatenate([idx, [0, n - 1]]).astype(np.int64))
    return idx[(idx >= 0) & (idx < n)]
