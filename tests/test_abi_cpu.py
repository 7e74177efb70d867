"""The C ABI without a GPU: libnrng.so loads, exports every function that
include/nrng.h declares, and its host-side validation returns the documented
status before anything is enqueued (only fake, never-dereferenced pointers
are passed, and only to calls that reject them on the host)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1004_3105_gb300 import _lib
from paper_1004_3105_gb300.nrng import STREAM_DESC

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "nrng.h")


@pytest.fixture(scope="module")
def lib():
    return _lib.load(build_if_missing=True)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nrng_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"
    assert lib.nrng_abi_version() == 1


def test_status_strings(lib):
    for code, name in _lib.STATUS.items():
        assert lib.nrng_status_string(code).decode().startswith(name)
    assert lib.nrng_status_string(99).decode() == "NRNG_ERR_UNKNOWN"


FAKE = ctypes.c_void_p(0x100000)       # 256-byte aligned, never dereferenced
ODD = ctypes.c_void_p(0x100001)


def test_boxmuller_validation(lib):
    f = lib.nrng_boxmuller
    assert f(None, -1, 0.0, 1.0, 1, 0, 0, 0, None) == _lib.ERR_INVALID_VALUE
    assert f(None, 5, 0.0, 1.0, 1, 0, 0, 0, None) == _lib.ERR_INVALID_VALUE
    assert f(FAKE, 5, 0.0, -1.0, 1, 0, 0, 0, None) == _lib.ERR_INVALID_VALUE
    assert f(FAKE, 5, float("nan"), 1.0, 1, 0, 0, 0, None) == _lib.ERR_INVALID_VALUE
    assert f(FAKE, 5, 0.0, float("inf"), 1, 0, 0, 0, None) == _lib.ERR_INVALID_VALUE
    assert f(FAKE, 5, 0.0, 1.0, 1, 0, 3, 0, None) == _lib.ERR_INVALID_VALUE      # dtype
    assert f(FAKE, 5, 0.0, 1.0, 1, 0, 0, 3, None) == _lib.ERR_INVALID_VALUE      # mode (2 = B2 is valid)
    assert f(FAKE, 5, 0.0, 1.0, 1, 0, 0, -1, None) == _lib.ERR_INVALID_VALUE
    assert f(ODD, 5, 0.0, 1.0, 1, 0, 0, 0, None) == _lib.ERR_MISALIGNED
    assert f(ODD, 5, 0.0, 1.0, 1, 0, 1, 0, None) == _lib.ERR_MISALIGNED          # bf16 needs 2 bytes
    # ceil(9/4) = 3 blocks from 2^64 - 2 would pass 2^64
    assert f(FAKE, 9, 0.0, 1.0, 1, 2 ** 64 - 2, 0, 0, None) == _lib.ERR_COUNTER_OVERFLOW
    assert f(FAKE, 0, 0.0, 1.0, 1, 0, 0, 0, None) == _lib.OK                      # n = 0: no-op
    assert f(None, 0, 0.0, 1.0, 1, 0, 0, 0, None) == _lib.OK


def test_uniform_validation(lib):
    f = lib.nrng_uniform
    assert f(None, 3, 1, 0, None) == _lib.ERR_INVALID_VALUE
    assert f(ctypes.c_void_p(0x100002), 3, 1, 0, None) == _lib.ERR_MISALIGNED
    assert f(FAKE, 5, 1, 2 ** 64 - 1, None) == _lib.ERR_COUNTER_OVERFLOW
    assert f(FAKE, 0, 1, 0, None) == _lib.OK


def test_polar_workspace_and_validation(lib):
    b = ctypes.c_size_t(0)
    assert lib.nrng_polar_workspace_size(-1, ctypes.byref(b)) == _lib.ERR_INVALID_VALUE
    assert lib.nrng_polar_workspace_size(1 << 28, ctypes.byref(b)) == _lib.OK
    ws = b.value
    # one 8-byte word per tile of 4608 candidates (4 warps x 18 rows x 32 lanes
    # x 2) at the 0.78 budget + 64-byte header
    tiles = ((1 << 27) + 12 * (int(np.sqrt(1 << 27)) + 1) + 16) * 100
    tiles = (tiles + 4608 * 78 - 1) // (4608 * 78) + 1
    assert ws == (64 + 8 * tiles + 255) // 256 * 256
    blocks = ctypes.c_uint64(0)
    assert lib.nrng_polar_max_blocks(1 << 28, ctypes.byref(blocks)) == _lib.OK
    assert blocks.value == tiles * 2304
    # workspace too small / missing
    f = lib.nrng_polar
    assert f(FAKE, 100, 0.0, 1.0, 1, 0, 0, 0, FAKE, 8, None, None, None) == _lib.ERR_WORKSPACE
    assert f(FAKE, 100, 0.0, 1.0, 1, 0, 0, 0, None, 1 << 20, None, None, None) == _lib.ERR_WORKSPACE
    assert f(FAKE, 100, 0.0, -2.0, 1, 0, 0, 0, FAKE, 1 << 20, None, None, None) == _lib.ERR_INVALID_VALUE
    assert f(FAKE, 100, 0.0, 1.0, 1, 2 ** 64 - 5, 0, 0, FAKE, 1 << 20, None, None, None) == \
        _lib.ERR_COUNTER_OVERFLOW
    assert f(FAKE, 100, 0.0, 1.0, 1, 0, 0, 0, ctypes.c_void_p(0x100004), 1 << 20, None, None, None) == \
        _lib.ERR_MISALIGNED
    assert f(FAKE, (1 << 48) + 1, 0.0, 1.0, 1, 0, 0, 0, FAKE, 1 << 40, None, None, None) == \
        _lib.ERR_INVALID_VALUE


def test_tile_budget_integer_sqrt(lib):
    """The tile budget takes floor(sqrt(items)) in integers (a float root, one
    Newton step and exact corrections): around perfect squares, where a root
    one off would change the budget, the workspace sizes must follow the
    exact integer square root (items = ceil(n/2) for P, n for R)."""
    import math
    b = ctypes.c_size_t(0)
    ks = [1, 2, 3, 1000, 46340, 46341, 65535, 65536, 1 << 20, (1 << 23) - 1, 1 << 23, 3037000499 >> 8]
    for k in ks:
        for items in (k * k - 1, k * k, k * k + 1):
            if items < 1:
                continue
            n = 2 * items   # P: ceil(n/2) = items
            assert lib.nrng_polar_workspace_size(n, ctypes.byref(b)) == _lib.OK
            need = items + 12 * (math.isqrt(items) + 1) + 16
            tiles = (need * 100 + 4608 * 78 - 1) // (4608 * 78) + 1
            assert b.value == (64 + 8 * tiles + 255) // 256 * 256, (n, b.value)
            assert lib.nrng_ratio_workspace_size(items, ctypes.byref(b)) == _lib.OK
            tiles = (need * 100 + 3584 * 72 - 1) // (3584 * 72) + 1
            assert b.value == (64 + 8 * tiles + 255) // 256 * 256, (items, b.value)


def test_b3_validation(lib):
    f = lib.nrng_boxmuller_b3
    assert f(None, 5, 0.0, 1.0, 1, 0, 0, None) == _lib.ERR_INVALID_VALUE
    assert f(FAKE, -1, 0.0, 1.0, 1, 0, 0, None) == _lib.ERR_INVALID_VALUE
    assert f(FAKE, 5, 0.0, -1.0, 1, 0, 0, None) == _lib.ERR_INVALID_VALUE
    assert f(FAKE, 5, 0.0, 1.0, 1, 0, 7, None) == _lib.ERR_INVALID_VALUE
    assert f(ODD, 5, 0.0, 1.0, 1, 0, 2, None) == _lib.ERR_MISALIGNED
    # 9 outputs take 3 ceil(9/8) = 6 blocks: from 2^64 - 5 they would pass 2^64
    assert f(FAKE, 9, 0.0, 1.0, 1, 2 ** 64 - 5, 0, None) == _lib.ERR_COUNTER_OVERFLOW
    assert f(FAKE, 0, 0.0, 1.0, 1, 0, 0, None) == _lib.OK


def test_p2_validation(lib):
    f = lib.nrng_polar_p2
    assert f(FAKE, 100, 0.0, 1.0, 1, 0, 0, FAKE, 8, None, None, None) == _lib.ERR_WORKSPACE
    assert f(FAKE, 100, 0.0, 1.0, 1, 0, 0, None, 1 << 20, None, None, None) == _lib.ERR_WORKSPACE
    assert f(FAKE, 100, 0.0, 1.0, 1, 0, 9, FAKE, 1 << 20, None, None, None) == _lib.ERR_INVALID_VALUE
    assert f(FAKE, 100, 0.0, float("nan"), 1, 0, 0, FAKE, 1 << 20, None, None, None) == _lib.ERR_INVALID_VALUE
    assert f(FAKE, 100, 0.0, 1.0, 1, 2 ** 64 - 5, 0, FAKE, 1 << 20, None, None, None) == \
        _lib.ERR_COUNTER_OVERFLOW
    assert f(FAKE, 100, 0.0, 1.0, 1, 0, 0, FAKE, 1 << 20, ODD, None, None) == _lib.ERR_MISALIGNED
    assert f(None, 0, 0.0, 1.0, 1, 0, 0, None, 0, None, None, None) == _lib.OK


def test_ratio_workspace_and_validation(lib):
    b = ctypes.c_size_t(0)
    assert lib.nrng_ratio_workspace_size(-1, ctypes.byref(b)) == _lib.ERR_INVALID_VALUE
    n = 1 << 28
    assert lib.nrng_ratio_workspace_size(n, ctypes.byref(b)) == _lib.OK
    # one word per tile of 3584 candidates (4 warps x 14 rows x 32 lanes x 2)
    # at the 0.72 budget (acceptance sqrt(pi e)/4 = 0.7306)
    tiles = (n + 12 * (int(np.sqrt(n)) + 1) + 16) * 100
    tiles = (tiles + 3584 * 72 - 1) // (3584 * 72) + 1
    assert b.value == (64 + 8 * tiles + 255) // 256 * 256
    f = lib.nrng_ratio
    assert f(FAKE, 100, 0.0, 1.0, 1, 0, 0, 0, FAKE, 8, None, None, None) == _lib.ERR_WORKSPACE
    assert f(FAKE, 100, 0.0, 1.0, 1, 0, 0, 2, FAKE, 1 << 20, None, None, None) == _lib.ERR_INVALID_VALUE
    assert f(FAKE, 100, 0.0, 1.0, 1, 0, 3, 0, FAKE, 1 << 20, None, None, None) == _lib.ERR_INVALID_VALUE
    assert f(FAKE, 100, 0.0, -1.0, 1, 0, 0, 0, FAKE, 1 << 20, None, None, None) == _lib.ERR_INVALID_VALUE
    assert f(FAKE, 100, 0.0, 1.0, 1, 2 ** 64 - 5, 0, 0, FAKE, 1 << 20, None, None, None) == \
        _lib.ERR_COUNTER_OVERFLOW
    assert f(ODD, 100, 0.0, 1.0, 1, 0, 1, 0, FAKE, 1 << 20, None, None, None) == _lib.ERR_MISALIGNED
    assert f(FAKE, 100, 0.0, 1.0, 1, 0, 0, 0, FAKE, 1 << 20, None, ODD, None) == _lib.ERR_MISALIGNED
    assert f(FAKE, (1 << 48) + 1, 0.0, 1.0, 1, 0, 0, 0, FAKE, 1 << 40, None, None, None) == \
        _lib.ERR_INVALID_VALUE
    assert f(None, 0, 0.0, 1.0, 1, 0, 0, 0, None, 0, None, None, None) == _lib.OK


def _desc(ns, methods):
    d = np.zeros(len(ns), dtype=STREAM_DESC)
    d["n"] = ns
    d["offset"] = np.concatenate([[0], np.cumsum(ns)[:-1]])
    d["sigma"] = 1.0
    d["method"] = methods
    d["key"] = np.arange(len(ns))
    return d


def test_batched_workspace_size(lib):
    d = _desc([100, 1000, 0, 5000], [0, 1, 1, 1])
    b = ctypes.c_size_t(0)
    assert lib.nrng_batched_workspace_size(d.ctypes.data_as(ctypes.c_void_p), len(d), ctypes.byref(b)) == _lib.OK
    k = len(d)
    # header, slot bases (k + 1), completion flags, per-stream counts and
    # item bases (16 bytes each, from a 16-byte boundary), the setup's five
    # look-back words per 256 streams, then 256-aligned
    counts = (64 + (k + 1) * 8 + k * 4 + 15) // 16 * 16
    fixed = (counts + 16 * k + 16 * k + 5 * 8 * ((k + 255) // 256) + 255) // 256 * 256
    # most status slots plus item-table entries over the configurations (one
    # 8-byte entry each): a Polar stream's slots are its tile budget and its
    # items its expected tiles at acceptance pi/4 plus one overflow item; a B1
    # stream has no slots and one item per four tiles
    worst = 0
    for threads, bpt in [(128, 18), (128, 16), (128, 12), (128, 8), (256, 8), (128, 4), (256, 4)]:
        cand = 2 * threads * bpt
        s = 0
        for n, m in zip([100, 1000, 0, 5000], [0, 1, 1, 1]):
            if n == 0:
                continue
            if m == 0:
                s += (((n + 3) // 4) + 4 * threads * bpt - 1) // (4 * threads * bpt)
                continue
            npairs = (n + 1) // 2
            need = npairs + 12 * (int(np.sqrt(npairs)) + 1) + 16
            budget = (need * 100 + cand * 78 - 1) // (cand * 78) + 1
            primary = min(max(1, (npairs * 10000 + cand * 7854 - 1) // (cand * 7854)), budget)
            s += budget + primary + 1
        worst = max(worst, s)
    assert b.value == fixed + 8 * worst
    big = _desc([100, 2 ** 60 + 1], [0, 0])   # a stream beyond the element cap
    assert lib.nrng_batched_workspace_size(big.ctypes.data_as(ctypes.c_void_p), len(big),
                                           ctypes.byref(b)) == _lib.ERR_INVALID_VALUE
    f = lib.nrng_batched
    assert f(FAKE, FAKE, -1, 0, 0, FAKE, 1 << 20, None) == _lib.ERR_INVALID_VALUE
    assert f(FAKE, FAKE, 4, 0, 0, None, 1 << 20, None) == _lib.ERR_WORKSPACE
    assert f(FAKE, FAKE, 4, 0, 0, ctypes.c_void_p(0x100008), 1 << 20, None) == _lib.ERR_MISALIGNED
    assert f(FAKE, FAKE, 4, 0, 0, FAKE, 16, None) == _lib.ERR_WORKSPACE
    assert f(FAKE, FAKE, 0, 0, 0, FAKE, 16, None) == _lib.OK


def test_element_counts_above_2p60_rejected(lib):
    """Counts beyond 2^60 (where the size arithmetic could overflow int64)
    are rejected before anything is enqueued, up to INT64_MAX."""
    for n in (2 ** 60 + 1, 2 ** 63 - 1):
        assert lib.nrng_uniform(FAKE, n, 1, 0, None) == _lib.ERR_INVALID_VALUE
        assert lib.nrng_boxmuller(FAKE, n, 0.0, 1.0, 1, 0, 0, 0, None) == _lib.ERR_INVALID_VALUE
        assert lib.nrng_boxmuller_b3(FAKE, n, 0.0, 1.0, 1, 0, 0, None) == _lib.ERR_INVALID_VALUE
        assert lib.nrng_eval_points(0, 0, FAKE, n, 0.0, 1.0, FAKE, None, None) == _lib.ERR_INVALID_VALUE
        assert lib.nrng_reparam_fwd(FAKE, FAKE, FAKE, n, 1, 1, 1, 0, 0, None) == _lib.ERR_INVALID_VALUE
        assert lib.nrng_reparam_bwd(FAKE, FAKE, FAKE, n, 1, 1, 1, 0, 0, None) == _lib.ERR_INVALID_VALUE
    # at the cap the host checks pass on to the counter check
    assert lib.nrng_uniform(FAKE, 2 ** 60, 1, 2 ** 64 - 1, None) == _lib.ERR_COUNTER_OVERFLOW


def test_philox_ceiling_validation(lib):
    f = lib.nrng_philox_ceiling
    assert f(None, 16, 1, 0, None) == _lib.ERR_INVALID_VALUE
    assert f(FAKE, -1, 1, 0, None) == _lib.ERR_INVALID_VALUE
    assert f(ctypes.c_void_p(0x100002), 16, 1, 0, None) == _lib.ERR_MISALIGNED
    assert f(FAKE, 0, 1, 0, None) == _lib.OK
    # 32-bit indices only, and a low counter word that does not wrap
    assert f(FAKE, 2 ** 31 + 1, 1, 0, None) == _lib.ERR_NOT_SUPPORTED
    assert f(FAKE, 16, 1, 2 ** 32 - 8, None) == _lib.ERR_NOT_SUPPORTED


def test_reparam_validation(lib):
    f = lib.nrng_reparam_fwd
    assert f(FAKE, FAKE, FAKE, 12, 5, 1, 1, 0, 0, None) == _lib.ERR_INVALID_VALUE     # 5 does not divide 12
    assert f(FAKE, FAKE, FAKE, 12, 0, 1, 1, 0, 0, None) == _lib.ERR_INVALID_VALUE
    assert f(None, FAKE, FAKE, 12, 12, 1, 1, 0, 0, None) == _lib.ERR_INVALID_VALUE
    assert f(ODD, FAKE, FAKE, 12, 12, 1, 1, 0, 0, None) == _lib.ERR_MISALIGNED
    g = lib.nrng_reparam_bwd
    assert g(None, None, FAKE, 12, 12, 1, 1, 0, 0, None) == _lib.ERR_INVALID_VALUE
    assert g(None, FAKE, FAKE, 12, 12, 1, 1, 2 ** 64 - 1, 0, None) == _lib.ERR_COUNTER_OVERFLOW


def test_config_table(lib):
    n = lib.nrng_batched_config_count()
    assert n == 7
    t, b = ctypes.c_int32(0), ctypes.c_int32(0)
    seen = set()
    for c in range(n):
        assert lib.nrng_batched_config_info(c, ctypes.byref(t), ctypes.byref(b)) == _lib.OK
        seen.add((t.value, b.value))
        assert t.value % 32 == 0 and b.value % 2 == 0 and 2 * t.value * b.value <= 4608
    assert len(seen) == n
    assert lib.nrng_batched_config_info(n, ctypes.byref(t), ctypes.byref(b)) == _lib.ERR_INVALID_VALUE
    c = ctypes.c_int32(0)
    assert lib.nrng_batched_set_config(0, 1, 4) == _lib.OK
    assert lib.nrng_batched_get_config(0, 1, ctypes.byref(c)) == _lib.OK and c.value == 4
    assert lib.nrng_batched_set_config(0, 1, -1) == _lib.OK
    assert lib.nrng_batched_get_config(0, 1, ctypes.byref(c)) == _lib.OK and c.value == 0   # default 128 x 18
    assert lib.nrng_batched_set_config(0, 1, 99) == _lib.ERR_INVALID_VALUE


def test_eval_points_validation(lib):
    f = lib.nrng_eval_points
    assert f(7, 0, FAKE, 4, 0.0, 1.0, FAKE, None, None) == _lib.ERR_INVALID_VALUE      # kind
    assert f(5, 0, FAKE, 4, 0.0, 1.0, FAKE, None, None) == _lib.ERR_INVALID_VALUE
    assert f(-1, 0, FAKE, 4, 0.0, 1.0, FAKE, None, None) == _lib.ERR_INVALID_VALUE
    for kind in (1, 2, 3, 4):                                                           # B2 is a B1 mode
        assert f(kind, 2, FAKE, 4, 0.0, 1.0, FAKE, None, None) == _lib.ERR_INVALID_VALUE
    for kind in (2, 3, 4):
        assert f(kind, 0, None, 0, 0.0, 1.0, None, None, None) == _lib.OK
    assert f(0, 5, FAKE, 4, 0.0, 1.0, FAKE, None, None) == _lib.ERR_INVALID_VALUE
    assert f(0, 0, None, 4, 0.0, 1.0, FAKE, None, None) == _lib.ERR_INVALID_VALUE
    assert f(0, 0, FAKE, 4, 0.0, -1.0, FAKE, None, None) == _lib.ERR_INVALID_VALUE
    assert f(0, 0, ODD, 4, 0.0, 1.0, FAKE, None, None) == _lib.ERR_MISALIGNED
    assert f(1, 0, FAKE, 4, 0.0, 1.0, FAKE, ODD, None) == _lib.ERR_MISALIGNED
    assert f(0, 0, None, 0, 0.0, 1.0, None, None, None) == _lib.OK


def test_launch_failure_maps_to_err_cuda(lib):
    """With no usable GPU a launch fails inside the runtime: the call returns
    NRNG_ERR_CUDA instead of crashing.  (Runs only where there is no GPU: with
    one, the fake output pointer would be written.)"""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    assert lib.nrng_uniform(FAKE, 8, 1, 0, None) == _lib.ERR_CUDA
    assert lib.nrng_boxmuller(FAKE, 8, 0.0, 1.0, 1, 0, 0, 0, None) == _lib.ERR_CUDA


def test_force_config_env():
    """NRNG_FORCE_CONFIG replaces the default batched configuration (read once
    per process, so checked in a child)."""
    import subprocess
    import sys
    code = ("import ctypes; from paper_1004_3105_gb300 import _lib; lib = _lib.load(); c = ctypes.c_int32(-9); "
            "assert lib.nrng_batched_get_config(0, 0, ctypes.byref(c)) == 0; print(c.value)")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for env_val, want in (("4", 4), ("99", None), ("", None)):
        env = dict(os.environ, NRNG_FORCE_CONFIG=env_val)
        out = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True,
                             timeout=300)
        assert out.returncode == 0, out.stderr
        got = int(out.stdout.strip())
        assert got == (want if want is not None else 0), (env_val, got)

