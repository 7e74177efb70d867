"""Python binding of the C ABI (include/nrng.h), with the same names.

Each nrng_* function here takes torch tensors where the C call takes device
pointers, reads the element type from the output tensor and the stream from
torch's current CUDA stream, calls the C entry point of the same name and
raises NrngError on a non-OK status.  It marshals arguments only: every step
of the generators runs in libnrng.so's kernels, and there is no CPU path.
Reparam wraps nrng_reparam_fwd/bwd in a torch.autograd.Function.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from ._lib import NrngError, check, load

ACCURATE, FAST, B2 = 0, 1, 2
B1, POLAR = 0, 1
# kinds of nrng_eval_points (B1 and POLAR double as the first two)
POINTS_P2, POINTS_RATIO, POINTS_B3 = 2, 3, 4
_MODES = {"accurate": ACCURATE, "fast": FAST, "b2": B2, ACCURATE: ACCURATE, FAST: FAST, B2: B2}
_DTYPES = {torch.float32: 0, torch.bfloat16: 1, torch.float16: 2}

# nrng_stream_desc_t, field for field (48 bytes).
STREAM_DESC = np.dtype([("offset", "<i8"), ("n", "<i8"), ("mu", "<f4"), ("sigma", "<f4"),
                        ("key", "<u8"), ("counter", "<u8"), ("method", "<i4"), ("reserved", "<i4")])
assert STREAM_DESC.itemsize == 48


def _mode(mode) -> int:
    try:
        return _MODES[mode]
    except KeyError:
        raise ValueError(f"mode must be 'accurate', 'fast' or 'b2', got {mode!r}") from None


def _dtype(t: torch.Tensor) -> int:
    try:
        return _DTYPES[t.dtype]
    except KeyError:
        raise TypeError(f"output dtype must be float32, bfloat16 or float16, got {t.dtype}") from None


def _dev(t: torch.Tensor, name: str):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _u64(v: int) -> int:
    v = int(v)
    if v < 0 or v >= 1 << 64:
        raise ValueError(f"key/counter must be in [0, 2^64), got {v}")
    return v


# ------------------------------------------------------------ single streams
def nrng_uniform(out: torch.Tensor, key: int, counter: int, stream=None) -> None:
    """out[i] = (word i of the Philox stream >> 8) * 2^-24, float32."""
    if out.dtype != torch.float32:
        raise TypeError("nrng_uniform writes float32")
    check(load().nrng_uniform(_dev(out, "out"), out.numel(), _u64(key), _u64(counter), _stream(stream)),
          "nrng_uniform")


def nrng_philox_ceiling(out: torch.Tensor, nblocks: int, key: int, counter: int, stream=None) -> None:
    """Draws Philox blocks [counter, counter + nblocks) and stores the xor of
    all their words in out[0] (int32 or uint32 tensor): a measurement of the
    generator's rate with no output traffic."""
    if out.dtype not in (torch.int32, getattr(torch, "uint32", torch.int32)) or out.numel() < 1:
        raise TypeError("nrng_philox_ceiling writes one 32-bit word")
    check(load().nrng_philox_ceiling(_dev(out, "out"), int(nblocks), _u64(key), _u64(counter), _stream(stream)),
          "nrng_philox_ceiling")


def nrng_boxmuller(out: torch.Tensor, mu: float, sigma: float, key: int, counter: int,
                   mode="accurate", stream=None) -> None:
    """Algorithm B1 into `out` (float32, bfloat16 or float16)."""
    check(load().nrng_boxmuller(_dev(out, "out"), out.numel(), float(mu), float(sigma), _u64(key),
                                _u64(counter), _dtype(out), _mode(mode), _stream(stream)),
          "nrng_boxmuller")


def nrng_polar_workspace_size(n: int) -> int:
    b = ctypes.c_size_t(0)
    check(load().nrng_polar_workspace_size(int(n), ctypes.byref(b)), "nrng_polar_workspace_size")
    return int(b.value)


def nrng_polar_max_blocks(n: int) -> int:
    b = ctypes.c_uint64(0)
    check(load().nrng_polar_max_blocks(int(n), ctypes.byref(b)), "nrng_polar_max_blocks")
    return int(b.value)


def polar_workspace(n: int, device=None) -> torch.Tensor:
    """A device buffer of nrng_polar_workspace_size(n) bytes (uint8)."""
    return torch.empty(max(nrng_polar_workspace_size(n), 256), dtype=torch.uint8,
                       device=device or "cuda")


def nrng_polar(out: torch.Tensor, mu: float, sigma: float, key: int, counter: int, workspace: torch.Tensor,
               mode="accurate", next_counter: torch.Tensor = None, pair_candidate: torch.Tensor = None,
               stream=None) -> None:
    """Algorithm P with order-preserving compaction into `out`.

    workspace: uint8 CUDA tensor of at least nrng_polar_workspace_size(n) bytes.
    next_counter: optional int64/uint64 CUDA tensor of one element.
    pair_candidate: optional int64 CUDA tensor of ceil(n/2) elements.
    """
    n = out.numel()
    if next_counter is not None and (next_counter.numel() < 1 or next_counter.element_size() != 8):
        raise ValueError("next_counter must hold one 64-bit element")
    if pair_candidate is not None and (pair_candidate.dtype != torch.int64 or pair_candidate.numel() < (n + 1) // 2):
        raise ValueError("pair_candidate must be int64 with ceil(n/2) elements")
    check(load().nrng_polar(_dev(out, "out"), n, float(mu), float(sigma), _u64(key), _u64(counter), _dtype(out),
                            _mode(mode), _dev(workspace, "workspace"), workspace.numel() * workspace.element_size(),
                            _dev(next_counter, "next_counter"), _dev(pair_candidate, "pair_candidate"),
                            _stream(stream)),
          "nrng_polar")


def nrng_polar_twopass_workspace_size(n: int) -> int:
    b = ctypes.c_size_t(0)
    check(load().nrng_polar_twopass_workspace_size(int(n), ctypes.byref(b)), "nrng_polar_twopass_workspace_size")
    return int(b.value)


def nrng_polar_twopass(out: torch.Tensor, mu: float, sigma: float, key: int, counter: int, workspace: torch.Tensor,
                       mode="accurate", next_counter: torch.Tensor = None, pair_candidate: torch.Tensor = None,
                       stream=None) -> None:
    """nrng_polar's outputs by a count pass, a scan and a write pass.
    workspace: uint8 CUDA tensor of nrng_polar_twopass_workspace_size(n) bytes."""
    n = out.numel()
    if pair_candidate is not None and (pair_candidate.dtype != torch.int64 or pair_candidate.numel() < (n + 1) // 2):
        raise ValueError("pair_candidate must be int64 with ceil(n/2) elements")
    check(load().nrng_polar_twopass(_dev(out, "out"), n, float(mu), float(sigma), _u64(key), _u64(counter),
                                    _dtype(out), _mode(mode), _dev(workspace, "workspace"),
                                    workspace.numel() * workspace.element_size(), _dev(next_counter, "next_counter"),
                                    _dev(pair_candidate, "pair_candidate"), _stream(stream)),
          "nrng_polar_twopass")


def _check_next_counter(next_counter):
    if next_counter is not None and (next_counter.numel() < 1 or next_counter.element_size() != 8):
        raise ValueError("next_counter must hold one 64-bit element")


def _check_candidates(cand, need, name):
    if cand is not None and (cand.dtype != torch.int64 or cand.numel() < need):
        raise ValueError(f"{name} must be int64 with at least {need} elements")


def nrng_boxmuller_b3(out: torch.Tensor, mu: float, sigma: float, key: int, counter: int, stream=None) -> None:
    """Method B3: three uniforms per pair, h(v) for the radius, B2's sine and
    cosine; fills `out` (uses 3 ceil(n/8) Philox blocks)."""
    check(load().nrng_boxmuller_b3(_dev(out, "out"), out.numel(), float(mu), float(sigma), _u64(key),
                                   _u64(counter), _dtype(out), _stream(stream)),
          "nrng_boxmuller_b3")


def nrng_polar_p2(out: torch.Tensor, mu: float, sigma: float, key: int, counter: int, workspace: torch.Tensor,
                  next_counter: torch.Tensor = None, pair_candidate: torch.Tensor = None, stream=None) -> None:
    """Method P2: Algorithm P's candidates and accept order, radius from 1 - s.
    workspace: uint8 CUDA tensor of nrng_polar_workspace_size(n) bytes."""
    n = out.numel()
    _check_next_counter(next_counter)
    _check_candidates(pair_candidate, (n + 1) // 2, "pair_candidate")
    check(load().nrng_polar_p2(_dev(out, "out"), n, float(mu), float(sigma), _u64(key), _u64(counter), _dtype(out),
                               _dev(workspace, "workspace"), workspace.numel() * workspace.element_size(),
                               _dev(next_counter, "next_counter"), _dev(pair_candidate, "pair_candidate"),
                               _stream(stream)),
          "nrng_polar_p2")


def nrng_ratio_workspace_size(n: int) -> int:
    b = ctypes.c_size_t()
    check(load().nrng_ratio_workspace_size(int(n), ctypes.byref(b)), "nrng_ratio_workspace_size")
    return b.value


def ratio_workspace(n: int, device=None) -> torch.Tensor:
    """A device buffer of nrng_ratio_workspace_size(n) bytes (uint8)."""
    return torch.empty(max(nrng_ratio_workspace_size(n), 256), dtype=torch.uint8, device=device or "cuda")


def nrng_ratio(out: torch.Tensor, mu: float, sigma: float, key: int, counter: int, workspace: torch.Tensor,
               mode="accurate", next_counter: torch.Tensor = None, candidate: torch.Tensor = None,
               stream=None) -> None:
    """Algorithm R (ratio of uniforms), one value per accepted candidate, in order.
    candidate: optional int64 CUDA tensor of n elements (index of each output's candidate)."""
    n = out.numel()
    _check_next_counter(next_counter)
    _check_candidates(candidate, n, "candidate")
    check(load().nrng_ratio(_dev(out, "out"), n, float(mu), float(sigma), _u64(key), _u64(counter), _dtype(out),
                            _mode(mode), _dev(workspace, "workspace"), workspace.numel() * workspace.element_size(),
                            _dev(next_counter, "next_counter"), _dev(candidate, "candidate"), _stream(stream)),
          "nrng_ratio")


def nrng_eval_points(kind: int, points: torch.Tensor, mu: float = 0.0, sigma: float = 1.0, mode="accurate",
                     stream=None):
    """The per-pair transform at given inputs (diagnostics).  kind B1 and
    POINTS_RATIO: points is an [n, 2] uint32/int32 tensor of Philox words
    (wu, wv); POLAR and POINTS_P2: an [n, 2] int32 tensor of lattice
    coordinates (kx', ky'); POINTS_B3: an [n, 3] tensor of words (w1, w2, w3).
    Returns (values [n, 2] float32, accept [n] int32)."""
    width = 3 if kind == POINTS_B3 else 2
    if points.dim() != 2 or points.shape[1] != width or points.element_size() != 4:
        raise ValueError(f"points must be an [n, {width}] tensor of 32-bit words")
    pts = points.contiguous()
    n = pts.shape[0]
    out = torch.empty((n, 2), dtype=torch.float32, device=pts.device)
    acc = torch.empty(n, dtype=torch.int32, device=pts.device)
    check(load().nrng_eval_points(int(kind), _mode(mode), _dev(pts, "points"), n, float(mu), float(sigma),
                                  _dev(out, "out"), _dev(acc, "accept"), _stream(stream)),
          "nrng_eval_points")
    return out, acc


def nrng_polar_noalloc(out: torch.Tensor, mu: float, sigma: float, key: int, counter: int, mode="accurate",
                       next_counter: torch.Tensor = None, pair_candidate: torch.Tensor = None,
                       status: torch.Tensor = None, stream=None) -> None:
    """nrng_polar with the library's fixed device scratch instead of a caller
    workspace, for callers that cannot allocate device memory (n <= 2^28).
    status: optional int32 CUDA tensor that receives the device status word."""
    check(load().nrng_polar_noalloc(_dev(out, "out"), out.numel(), float(mu), float(sigma), _u64(key), _u64(counter),
                                    _dtype(out), _mode(mode), _dev(next_counter, "next_counter"),
                                    _dev(pair_candidate, "pair_candidate"), _dev(status, "status"), _stream(stream)),
          "nrng_polar_noalloc")


def nrng_get_status(workspace: torch.Tensor, stream=None) -> int:
    """The status word a workspace call left (synchronises the stream)."""
    v = ctypes.c_int32(0)
    check(load().nrng_get_status(_dev(workspace, "workspace"), _stream(stream), ctypes.byref(v)), "nrng_get_status")
    return int(v.value)


def raise_on_status(workspace: torch.Tensor, where: str = "", stream=None) -> None:
    st = nrng_get_status(workspace, stream)
    if st != 0:
        raise NrngError(st, where or "device status")


# ------------------------------------------------------------------ batched
def stream_descriptors(offset, n, mu, sigma, key, counter, method) -> np.ndarray:
    """Pack per-stream arrays into nrng_stream_desc_t records (host)."""
    k = len(n)
    d = np.zeros(k, dtype=STREAM_DESC)
    d["offset"], d["n"], d["mu"], d["sigma"] = offset, n, mu, sigma
    d["key"], d["counter"], d["method"] = key, counter, method
    return d


def nrng_batched_workspace_size(desc: np.ndarray) -> int:
    desc = np.ascontiguousarray(desc, dtype=STREAM_DESC)
    b = ctypes.c_size_t(0)
    check(load().nrng_batched_workspace_size(desc.ctypes.data_as(ctypes.c_void_p), len(desc), ctypes.byref(b)),
          "nrng_batched_workspace_size")
    return int(b.value)


def descriptors_to_device(desc: np.ndarray, device=None) -> torch.Tensor:
    raw = np.ascontiguousarray(desc, dtype=STREAM_DESC).view(np.uint8)
    return torch.from_numpy(raw.copy()).to(device or "cuda")


def nrng_batched(out: torch.Tensor, desc_dev: torch.Tensor, k: int, workspace: torch.Tensor, mode="accurate",
                 stream=None) -> None:
    """k streams (descriptors already on the device) in one persistent launch."""
    check(load().nrng_batched(_dev(out, "out"), _dev(desc_dev, "desc"), int(k), _dtype(out), _mode(mode),
                              _dev(workspace, "workspace"), workspace.numel() * workspace.element_size(),
                              _stream(stream)),
          "nrng_batched")


def nrng_batched_config_count() -> int:
    return int(load().nrng_batched_config_count())


def nrng_batched_config_info(config: int):
    t, b = ctypes.c_int32(0), ctypes.c_int32(0)
    check(load().nrng_batched_config_info(int(config), ctypes.byref(t), ctypes.byref(b)), "config_info")
    return int(t.value), int(b.value)


def nrng_batched_set_config(dtype: torch.dtype, mode, config: int) -> None:
    check(load().nrng_batched_set_config(_DTYPES[dtype], _mode(mode), int(config)), "nrng_batched_set_config")


def nrng_batched_get_config(dtype: torch.dtype, mode) -> int:
    c = ctypes.c_int32(0)
    check(load().nrng_batched_get_config(_DTYPES[dtype], _mode(mode), ctypes.byref(c)), "nrng_batched_get_config")
    return int(c.value)


def nrng_batched_autotune(out: torch.Tensor, desc_dev: torch.Tensor, k: int, workspace: torch.Tensor,
                          mode="accurate", reps: int = 3, stream=None):
    """Times every compiled configuration, pins the fastest; returns (config, ms)."""
    c, ms = ctypes.c_int32(-1), ctypes.c_float(0.0)
    check(load().nrng_batched_autotune(_dev(out, "out"), _dev(desc_dev, "desc"), int(k), _dtype(out), _mode(mode),
                                       _dev(workspace, "workspace"), workspace.numel() * workspace.element_size(),
                                       int(reps), _stream(stream), ctypes.byref(c), ctypes.byref(ms)),
          "nrng_batched_autotune")
    return int(c.value), float(ms.value)


class BatchedGraph:
    """One nrng_batched call captured into a CUDA graph (nrng_batched_graph_create)."""

    def __init__(self, out, desc_dev, k, workspace, mode="accurate", stream=None):
        self._keep = (out, desc_dev, workspace)
        self._stream = stream or torch.cuda.Stream()
        h = ctypes.c_void_p(None)
        with torch.cuda.stream(self._stream):
            check(load().nrng_batched_graph_create(
                _dev(out, "out"), _dev(desc_dev, "desc"), int(k), _dtype(out), _mode(mode),
                _dev(workspace, "workspace"), workspace.numel() * workspace.element_size(),
                ctypes.c_void_p(self._stream.cuda_stream), ctypes.byref(h)), "nrng_batched_graph_create")
        self._h = h

    def launch(self, stream=None) -> None:
        check(load().nrng_graph_launch(self._h, _stream(stream)), "nrng_graph_launch")

    def close(self) -> None:
        if self._h is not None and self._h.value:
            load().nrng_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ reparam
def broadcast_layout(param_shape, out_shape):
    """(m, inner) of nrng_reparam_*: element i of the output uses parameter
    (i / inner) mod m.  The parameter's non-unit dims, after left-padding its
    shape with ones, must be one contiguous run equal to the output's dims."""
    out_shape = tuple(out_shape)
    ps = (1,) * (len(out_shape) - len(param_shape)) + tuple(param_shape)
    if len(ps) != len(out_shape):
        raise ValueError(f"parameter shape {tuple(param_shape)} has more dims than {out_shape}")
    nz = [i for i, d in enumerate(ps) if d != 1]
    if not nz:
        return 1, 1
    a, b = nz[0], nz[-1] + 1
    if any(ps[i] != out_shape[i] for i in range(a, b)):
        raise ValueError(f"parameter shape {tuple(param_shape)} does not broadcast to {out_shape} "
                         "along one contiguous run of dims")
    m = int(np.prod(out_shape[a:b]))
    inner = int(np.prod(out_shape[b:])) if b < len(out_shape) else 1
    return m, inner


def nrng_reparam_fwd(x: torch.Tensor, mu: torch.Tensor, sigma: torch.Tensor, key: int, counter: int,
                     mode="accurate", stream=None) -> None:
    """x = mu + sigma * z, z the B1 stream of (key, counter); mu and sigma share one shape."""
    if mu.shape != sigma.shape:
        raise ValueError("mu and sigma must have the same shape")
    if x.dtype != torch.float32 or mu.dtype != torch.float32 or sigma.dtype != torch.float32:
        raise TypeError("reparam tensors are float32")
    m, inner = broadcast_layout(mu.shape, x.shape)
    check(load().nrng_reparam_fwd(_dev(x, "x"), _dev(mu, "mu"), _dev(sigma, "sigma"), x.numel(), m, inner,
                                  _u64(key), _u64(counter), _mode(mode), _stream(stream)),
          "nrng_reparam_fwd")


def nrng_reparam_bwd(dmu, dsigma: torch.Tensor, g: torch.Tensor, key: int, counter: int,
                     mode="accurate", stream=None) -> None:
    """dmu = sum g, dsigma = sum g z over each parameter's elements (z regenerated)."""
    if g.dtype != torch.float32 or dsigma.dtype != torch.float32:
        raise TypeError("reparam tensors are float32")
    m, inner = broadcast_layout(dsigma.shape, g.shape)
    check(load().nrng_reparam_bwd(_dev(dmu, "dmu"), _dev(dsigma, "dsigma"), _dev(g, "g"), g.numel(), m, inner,
                                  _u64(key), _u64(counter), _mode(mode), _stream(stream)),
          "nrng_reparam_bwd")


class Reparam(torch.autograd.Function):
    """x = mu + sigma * z with z ~ N(0, 1) drawn by B1 from (key, counter).

    Nothing is saved for backward but the generator state: backward
    regenerates z from (key, counter) inside nrng_reparam_bwd.
    Usage: x = Reparam.apply(mu, sigma, shape, key, counter, mode)."""

    @staticmethod
    def forward(ctx, mu, sigma, shape, key, counter, mode="accurate"):
        mu_c, sigma_c = mu.contiguous(), sigma.contiguous()
        x = torch.empty(tuple(shape), dtype=torch.float32, device=mu.device)
        nrng_reparam_fwd(x, mu_c, sigma_c, key, counter, mode)
        ctx.key, ctx.counter, ctx.mode = int(key), int(counter), mode
        ctx.param_shape = mu.shape
        return x

    @staticmethod
    def backward(ctx, g):
        g = g.contiguous().float()
        need_mu, need_sigma = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        dsigma = torch.empty(ctx.param_shape, dtype=torch.float32, device=g.device)
        dmu = torch.empty_like(dsigma) if need_mu else None
        nrng_reparam_bwd(dmu, dsigma, g, ctx.key, ctx.counter, ctx.mode)
        return dmu, (dsigma if need_sigma else None), None, None, None, None
