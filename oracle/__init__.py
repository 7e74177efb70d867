"""FP64 CPU oracle for Brent's B1 (Box-Muller) and P (Polar) normal generators.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(the CUDA library and its binding) never does.  The arithmetic lives in
``nrng_oracle.c`` (plain single-threaded C, double precision); this module only
compiles it with gcc and marshals numpy arrays through ctypes.

Functions and the passages they follow (paper: Brent, TR-CS-93-04, 1993):
  philox4x32_10, philox_blocks   Philox-4x32-10 (Salmon et al., SC'11)
  uniform                        Sec. 2, uniforms on [0,1), note a
  boxmuller, boxmuller_at,       Sec. 2, Algorithm B1 (steps 1-3, notes a-b)
  b1_points
  polar, polar_candidates,       Sec. 2, Algorithm P (steps 1-4), rejected
  polar_points, polar_at,        pairs compressed in candidate order (Sec. 4)
  polar_accept_points
  lattice_accept_count           exact acceptance count of P's step 3
  batched                        independent B1/P streams
  b3, b3_points                  Sec. 3, Method B3 (exact function for h)
  polar_p2, p2_points            Sec. 4, Method P2 (step 4a, exact function for h)
  ratio, ratio_candidates,       Sec. 5, Algorithm R (ratio-of-uniforms region)
  ratio_at, ratio_points
  reparam_fwd, reparam_bwd       x = mu + sigma z with z from B1, and its
                                 gradients (an add-on; no counterpart in the paper)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nrng_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libnrng_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile nrng_oracle.c into a shared library with gcc; returns its path."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            os.makedirs(os.path.dirname(_LIB), exist_ok=True)
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                                   "-fno-fast-math", "-ffp-contract=off",
                                   "-D_DEFAULT_SOURCE", _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    i64, u64, i32, f64 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double
    sig = {
        "orc_philox4x32_10": (None, [P, P, P]),
        "orc_philox_blocks": (None, [P, i64, u64, u64]),
        "orc_uniform": (None, [P, i64, u64, u64]),
        "orc_boxmuller": (None, [P, i64, f64, f64, u64, u64]),
        "orc_boxmuller_at": (None, [P, P, i64, f64, f64, u64, u64]),
        "orc_b1_points": (None, [P, P, P, i64, f64, f64]),
        "orc_polar": (i64, [P, i64, f64, f64, u64, u64, P, P]),
        "orc_polar_candidates": (None, [P, P, P, i64, u64, u64]),
        "orc_polar_points": (None, [P, P, P, i64, f64, f64]),
        "orc_polar_accept_points": (None, [P, P, P, i64]),
        "orc_polar_at": (None, [P, P, i64, f64, f64, u64, u64]),
        "orc_lattice_accept_count": (i64, []),
        "orc_lattice_accept_count_h": (i64, [i64]),
        "orc_batched": (None, [P, i32, P, P, P, P, P, P, P]),
        "orc_b3": (None, [P, i64, f64, f64, u64, u64]),
        "orc_b3_points": (None, [P, P, P, P, i64, f64, f64]),
        "orc_p2_points": (None, [P, P, P, i64, f64, f64]),
        "orc_ratio_points": (None, [P, P, P, P, i64, f64, f64]),
        "orc_polar_p2": (i64, [P, i64, f64, f64, u64, u64, P, P]),
        "orc_ratio": (i64, [P, i64, f64, f64, u64, u64, P, P]),
        "orc_ratio_candidates": (None, [P, i64, u64, u64]),
        "orc_ratio_at": (None, [P, P, i64, f64, f64, u64, u64]),
        "orc_reparam_fwd": (None, [P, P, P, i64, i64, i64, u64, u64]),
        "orc_reparam_bwd": (None, [P, P, P, i64, i64, i64, u64, u64]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _u64(v: int) -> int:
    return int(v) & 0xFFFFFFFFFFFFFFFF


def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block for a 4-word counter and a 2-word key."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def philox_blocks(nblocks: int, key: int, counter: int) -> np.ndarray:
    """Words of blocks counter .. counter+nblocks-1, shape [nblocks, 4]."""
    out = np.zeros((nblocks, 4), dtype=np.uint32)
    _load().orc_philox_blocks(_ptr(out), nblocks, _u64(key), _u64(counter))
    return out


def uniform(n: int, key: int, counter: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.float64)
    _load().orc_uniform(_ptr(out), n, _u64(key), _u64(counter))
    return out


def boxmuller(n: int, mu: float, sigma: float, key: int, counter: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.float64)
    _load().orc_boxmuller(_ptr(out), n, float(mu), float(sigma), _u64(key), _u64(counter))
    return out


def boxmuller_at(idx, mu: float, sigma: float, key: int, counter: int) -> np.ndarray:
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros(idx.size, dtype=np.float64)
    _load().orc_boxmuller_at(_ptr(out), _ptr(idx), idx.size, float(mu), float(sigma),
                             _u64(key), _u64(counter))
    return out


def b1_points(u, v, mu: float, sigma: float) -> np.ndarray:
    """Steps 2-3 of B1 at given uniforms (u, v), shape [m, 2] = (x, y)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros((u.size, 2), dtype=np.float64)
    _load().orc_b1_points(_ptr(out), _ptr(u), _ptr(v), u.size, float(mu), float(sigma))
    return out


def polar(n: int, mu: float, sigma: float, key: int, counter: int):
    """Returns (out[n], pair_candidate[ceil(n/2)], next_counter, candidates examined)."""
    npairs = (n + 1) // 2
    out = np.zeros(n, dtype=np.float64)
    cand = np.zeros(npairs, dtype=np.int64)
    nxt = np.zeros(1, dtype=np.uint64)
    ncand = _load().orc_polar(_ptr(out), n, float(mu), float(sigma), _u64(key), _u64(counter),
                              _ptr(cand), _ptr(nxt))
    return out, cand, int(nxt[0]), int(ncand)


def polar_candidates(ncand: int, key: int, counter: int, coords: bool = True):
    """(accept[ncand] uint8, kx'[ncand], ky'[ncand]) for candidates 0 .. ncand-1
    (kx', ky' are None when coords is False)."""
    acc = np.zeros(ncand, dtype=np.uint8)
    kx = np.zeros(ncand, dtype=np.int32) if coords else None
    ky = np.zeros(ncand, dtype=np.int32) if coords else None
    _load().orc_polar_candidates(_ptr(acc), _ptr(kx), _ptr(ky), ncand, _u64(key), _u64(counter))
    return acc, kx, ky


def polar_points(kx, ky, mu: float, sigma: float) -> np.ndarray:
    """Step 4 at given lattice points, shape [m, 2]; NaN where step 3 rejects."""
    kx = np.ascontiguousarray(kx, dtype=np.int32)
    ky = np.ascontiguousarray(ky, dtype=np.int32)
    out = np.zeros((kx.size, 2), dtype=np.float64)
    _load().orc_polar_points(_ptr(out), _ptr(kx), _ptr(ky), kx.size, float(mu), float(sigma))
    return out


def polar_accept_points(kx, ky) -> np.ndarray:
    """Step 3's accept bit (uint8) at given lattice points."""
    kx = np.ascontiguousarray(kx, dtype=np.int32)
    ky = np.ascontiguousarray(ky, dtype=np.int32)
    acc = np.zeros(kx.size, dtype=np.uint8)
    _load().orc_polar_accept_points(_ptr(acc), _ptr(kx), _ptr(ky), kx.size)
    return acc


def polar_at(cand, mu: float, sigma: float, key: int, counter: int) -> np.ndarray:
    """Step 4 at given candidate indices of a stream, shape [m, 2]."""
    cand = np.ascontiguousarray(cand, dtype=np.int64)
    out = np.zeros((cand.size, 2), dtype=np.float64)
    _load().orc_polar_at(_ptr(out), _ptr(cand), cand.size, float(mu), float(sigma),
                         _u64(key), _u64(counter))
    return out


def lattice_accept_count(half_width: int = None) -> int:
    """Accepted points of step 3 on the lattice of half-width H (default the
    generator's 2^23): #{(a, b) in [-H, H)^2 : 0 < a^2 + b^2 < H^2}."""
    if half_width is None:
        return int(_load().orc_lattice_accept_count())
    return int(_load().orc_lattice_accept_count_h(int(half_width)))


def b3(n: int, mu: float, sigma: float, key: int, counter: int) -> np.ndarray:
    """Method B3 (Sec. 3) with the exact sqrt(-ln(1-u)); n outputs."""
    out = np.zeros(n, dtype=np.float64)
    _load().orc_b3(_ptr(out), n, float(mu), float(sigma), _u64(key), _u64(counter))
    return out


def b3_points(u1, u2, u3, mu: float, sigma: float) -> np.ndarray:
    """Method B3's pair at given uniforms, shape [m, 2]."""
    u1, u2, u3 = (np.ascontiguousarray(a, dtype=np.float64) for a in (u1, u2, u3))
    out = np.zeros((u1.size, 2), dtype=np.float64)
    _load().orc_b3_points(_ptr(out), _ptr(u1), _ptr(u2), _ptr(u3), u1.size, float(mu), float(sigma))
    return out


def p2_points(kx, ky, mu: float, sigma: float) -> np.ndarray:
    """Method P2's step 4a at given accepted lattice points, shape [m, 2]."""
    kx = np.ascontiguousarray(kx, dtype=np.int32)
    ky = np.ascontiguousarray(ky, dtype=np.int32)
    out = np.zeros((kx.size, 2), dtype=np.float64)
    _load().orc_p2_points(_ptr(out), _ptr(kx), _ptr(ky), kx.size, float(mu), float(sigma))
    return out


def polar_p2(n: int, mu: float, sigma: float, key: int, counter: int):
    """Method P2 (Sec. 4, step 4a); returns (out, pair_candidate, next_counter, candidates)."""
    npairs = (n + 1) // 2
    out = np.zeros(n, dtype=np.float64)
    cand = np.zeros(npairs, dtype=np.int64)
    nxt = np.zeros(1, dtype=np.uint64)
    nc = _load().orc_polar_p2(_ptr(out), n, float(mu), float(sigma), _u64(key), _u64(counter), _ptr(cand),
                              _ptr(nxt))
    return out, cand, int(nxt[0]), int(nc)


def ratio(n: int, mu: float, sigma: float, key: int, counter: int):
    """Algorithm R (Sec. 5); returns (out, candidate per output, next_counter, candidates)."""
    out = np.zeros(n, dtype=np.float64)
    cand = np.zeros(n, dtype=np.int64)
    nxt = np.zeros(1, dtype=np.uint64)
    nc = _load().orc_ratio(_ptr(out), n, float(mu), float(sigma), _u64(key), _u64(counter), _ptr(cand), _ptr(nxt))
    return out, cand, int(nxt[0]), int(nc)


def ratio_candidates(ncand: int, key: int, counter: int) -> np.ndarray:
    acc = np.zeros(ncand, dtype=np.uint8)
    _load().orc_ratio_candidates(_ptr(acc), ncand, _u64(key), _u64(counter))
    return acc


def ratio_at(cand, mu: float, sigma: float, key: int, counter: int) -> np.ndarray:
    cand = np.ascontiguousarray(cand, dtype=np.int64)
    out = np.zeros(cand.size, dtype=np.float64)
    _load().orc_ratio_at(_ptr(out), _ptr(cand), cand.size, float(mu), float(sigma), _u64(key), _u64(counter))
    return out


def ratio_points(u, v, mu: float, sigma: float):
    """Algorithm R's steps 2-4 at given uniforms; returns (accept uint8 [m],
    values [m], meaningful where accepted)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros(u.size, dtype=np.float64)
    acc = np.zeros(u.size, dtype=np.uint8)
    _load().orc_ratio_points(_ptr(out), _ptr(acc), _ptr(u), _ptr(v), u.size, float(mu), float(sigma))
    return acc, out


def batched(total: int, desc: dict) -> np.ndarray:
    """desc: dict of arrays offset, n, mu, sigma, key, counter, method (length k)."""
    k = len(desc["n"])
    out = np.full(total, np.nan, dtype=np.float64)
    arr = {
        "offset": np.ascontiguousarray(desc["offset"], dtype=np.int64),
        "n": np.ascontiguousarray(desc["n"], dtype=np.int64),
        "mu": np.ascontiguousarray(desc["mu"], dtype=np.float32),
        "sigma": np.ascontiguousarray(desc["sigma"], dtype=np.float32),
        "key": np.ascontiguousarray(desc["key"], dtype=np.uint64),
        "counter": np.ascontiguousarray(desc["counter"], dtype=np.uint64),
        "method": np.ascontiguousarray(desc["method"], dtype=np.int32),
    }
    _load().orc_batched(_ptr(out), k, *(_ptr(arr[f]) for f in
                        ("offset", "n", "mu", "sigma", "key", "counter", "method")))
    return out


def reparam_fwd(mu, sigma, n: int, inner: int, key: int, counter: int) -> np.ndarray:
    mu = np.ascontiguousarray(mu, dtype=np.float32).ravel()
    sigma = np.ascontiguousarray(sigma, dtype=np.float32).ravel()
    out = np.zeros(n, dtype=np.float64)
    _load().orc_reparam_fwd(_ptr(out), _ptr(mu), _ptr(sigma), n, mu.size, inner,
                            _u64(key), _u64(counter))
    return out


def reparam_bwd(g, m: int, inner: int, key: int, counter: int):
    """Returns (dmu[m], dsigma[m]) in FP64."""
    g = np.ascontiguousarray(g, dtype=np.float32).ravel()
    dmu = np.zeros(m, dtype=np.float64)
    dsig = np.zeros(m, dtype=np.float64)
    _load().orc_reparam_bwd(_ptr(dmu), _ptr(dsig), _ptr(g), g.size, m, inner,
                            _u64(key), _u64(counter))
    return dmu, dsig
