"""Tolerances and comparison helpers for the GPU parity tests.

Floating-point bar (per output, in output units):
  |x_gpu - x_ref| <= tol * sigma * max(1, |z_ref|) + ulp32(x_ref) / 2 [+ ulp_fmt(x_ref)]
with z_ref = (x_ref - mu) / sigma, tol = 4e-6 on the accurate path and 2e-5 on
the fast path (absolute in z, relative beyond |z| = 1), half an fp32 ulp for
the final rounding of mu + sigma z, and one ulp of bf16/fp16 for the
round-to-nearest-even of the fp32 result into a 16-bit output.
"""
import math

import numpy as np
import torch

TOL = {"accurate": 4e-6, "fast": 2e-5}
FMT_BITS = {torch.float32: None, torch.bfloat16: 8, torch.float16: 11}


def ulp_fmt(x: np.ndarray, dtype) -> np.ndarray:
    """One ulp of `dtype` at |x| (fp16 includes its subnormal spacing)."""
    ax = np.abs(x).astype(np.float64)
    if dtype == torch.float32:
        return np.spacing(ax.astype(np.float32)).astype(np.float64)
    p = FMT_BITS[dtype]
    e = np.floor(np.log2(np.maximum(ax, 1e-300)))
    if dtype == torch.float16:
        e = np.maximum(e, -14.0)
    return np.exp2(e - (p - 1))


def bound(ref: np.ndarray, mu: float, sigma: float, mode: str, dtype) -> np.ndarray:
    z = (ref - mu) / sigma if sigma > 0 else np.zeros_like(ref)
    b = TOL[mode] * sigma * np.maximum(1.0, np.abs(z)) + 0.5 * ulp_fmt(ref, torch.float32)
    if dtype != torch.float32:
        b = b + ulp_fmt(ref, dtype)
    return b


def assert_close(gpu: torch.Tensor, ref: np.ndarray, mu: float, sigma: float, mode: str, what: str = ""):
    got = gpu.detach().float().cpu().numpy().astype(np.float64)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    if got.size == 0:
        return 0.0
    err = np.abs(got - ref)
    b = bound(ref, mu, sigma, mode, gpu.dtype)
    bad = np.nonzero(~(err <= b))[0]
    if bad.size:
        i = bad[0]
        raise AssertionError(
            f"{what}: {bad.size} of {got.size} outside tolerance; first at {i}: gpu={got[i]!r} "
            f"ref={ref[i]!r} err={err[i]:.3e} bound={b[i]:.3e}")
    z = np.maximum(1.0, np.abs((ref - mu) / sigma)) if sigma > 0 else 1.0
    return float(np.max(err / (sigma * z))) if sigma > 0 else float(np.max(err))


def sync():
    torch.cuda.synchronize()


def canary_tensor(n: int, dtype, pad: int = 64, offset: int = 0, device="cuda"):
    """A buffer of offset + n + pad elements filled with a sentinel; returns
    (whole, view of n elements starting at offset)."""
    whole = torch.full((offset + n + pad,), -12345.0, dtype=dtype, device=device)
    return whole, whole[offset:offset + n]


def assert_canary(whole: torch.Tensor, offset: int, n: int):
    w = whole.float().cpu().numpy()
    sentinel = float(torch.tensor(-12345.0, dtype=whole.dtype).float())
    assert np.all(w[:offset] == sentinel), "write before the output"
    assert np.all(w[offset + n:] == sentinel), "write past the output"


def z_bins(ref: np.ndarray, got: np.ndarray, mu: float, sigma: float):
    """Max absolute and relative error per |z| bin [0,1), ..., [5,6), [6, inf)."""
    z = np.abs((ref - mu) / sigma)
    err = np.abs(got - ref)
    rel = err / np.maximum(np.abs(ref), 1e-30)
    rows = []
    edges = [0, 1, 2, 3, 4, 5, 6, math.inf]
    for lo, hi in zip(edges[:-1], edges[1:]):
        m = (z >= lo) & (z < hi)
        if m.any():
            rows.append((lo, hi, int(m.sum()), float(err[m].max()), float(rel[m].max()),
                         float((err[m] / sigma).max())))
        else:
            rows.append((lo, hi, 0, 0.0, 0.0, 0.0))
    return rows


def record_error_table(what: str, gpu: torch.Tensor, ref: np.ndarray, mu: float, sigma: float, n_total: int):
    """Appends the |z|-binned error rows of one variant to the JSON-lines file
    named by NRNG_ERROR_TABLE, when that variable is set (the precision-sweep
    error table); a no-op otherwise."""
    import json
    import os
    path = os.environ.get("NRNG_ERROR_TABLE")
    if not path:
        return
    got = gpu.detach().float().cpu().numpy().astype(np.float64)
    rows = z_bins(ref, got, mu, sigma)
    with open(path, "a") as f:
        f.write(json.dumps({"variant": what, "sampled": int(got.size), "of": int(n_total), "mu": mu,
                            "sigma": sigma, "bins": rows}) + "\n")

