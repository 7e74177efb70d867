"""nrng_polar_noalloc, the Polar entry point for callers that cannot allocate
device memory (a host application that owns the whole device budget, or a
loop that must not call cudaMalloc because it can synchronise the device).
Called through the C ABI, it must give what nrng_polar gives with a caller
workspace, on two calls in a row that share its fixed scratch array, and it
must refuse an n larger than the array can serve.  This file is collected
last and needs no state from the other tests."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1004_3105_gb300 as nr
from gpu_helpers import assert_close
from paper_1004_3105_gb300 import _lib

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _run_both(lib, n, mu, sigma, key, counter, mode, dtype, check_oracle=True, candidates=True):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    dt = {torch.float32: 0, torch.bfloat16: 1, torch.float16: 2}[dtype]
    md = {"accurate": 0, "fast": 1}[mode]
    npairs = (n + 1) // 2
    # the existing entry point, with a workspace the caller allocated
    ref = torch.empty(n, dtype=dtype, device="cuda")
    ws = torch.empty(nr.nrng_polar_workspace_size(n), dtype=torch.uint8, device="cuda")
    ref_next = torch.zeros(1, dtype=torch.int64, device="cuda")
    ref_cand = torch.empty(npairs, dtype=torch.int64, device="cuda") if candidates else None
    assert lib.nrng_polar(_p(ref), n, mu, sigma, key, counter, dt, md, _p(ws), ws.numel(), _p(ref_next),
                          _p(ref_cand), stream) == _lib.OK
    st = ctypes.c_int32(-1)
    assert lib.nrng_get_status(_p(ws), stream, ctypes.byref(st)) == _lib.OK and st.value == 0
    # the no-allocation entry point
    out = torch.empty(n, dtype=dtype, device="cuda")
    nxt = torch.zeros(1, dtype=torch.int64, device="cuda")
    cand = torch.empty(npairs, dtype=torch.int64, device="cuda") if candidates else None
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    assert lib.nrng_polar_noalloc(_p(out), n, mu, sigma, key, counter, dt, md, _p(nxt), _p(cand), _p(status),
                                  stream) == _lib.OK
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    if candidates:
        assert torch.equal(cand, ref_cand)
    assert int(nxt.item()) == int(ref_next.item())
    # the same kernel on the same inputs: the outputs are identical bit for bit
    assert torch.equal(out.view(torch.int16 if dtype != torch.float32 else torch.int32),
                       ref.view(torch.int16 if dtype != torch.float32 else torch.int32))
    if check_oracle:
        want, want_cand, want_next, _ = oracle.polar(n, mu, sigma, key, counter)
        if candidates:
            np.testing.assert_array_equal(cand.cpu().numpy(), want_cand)
        assert int(nxt.item()) == int(want_next)
        assert_close(out, want, mu, sigma, mode, f"noalloc n={n} vs oracle")


def test_noalloc_matches_workspace_entry_point_twice():
    lib = _lib.load()
    # two calls in a row on the shared scratch: a large stream, then a short
    # one with other parameters (stale tile words from the first would corrupt
    # the second if the array were not cleared)
    _run_both(lib, (1 << 22) + 1, 0.0, 1.0, 0x5EED0001, 0, "accurate", torch.float32)
    _run_both(lib, 100003, 1.5, 0.25, 77, 1 << 33, "fast", torch.bfloat16)


def test_noalloc_at_its_largest_n():
    # n = 2^28, the largest n the fixed array serves, is accepted and equals
    # nrng_polar (values bit for bit, next counter); the oracle check of this
    # size lives in the full-size tests of nrng_polar
    lib = _lib.load()
    _run_both(lib, 1 << 28, 0.0, 1.0, 0x5EED0001, 0, "accurate", torch.float32, check_oracle=False,
              candidates=False)
    torch.cuda.empty_cache()


def test_noalloc_n_zero():
    # n = 0 enqueues no generation: the status is OK and the next counter is
    # the given counter
    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = torch.empty(1, dtype=torch.float32, device="cuda")
    nxt = torch.full((1,), 7, dtype=torch.int64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    assert lib.nrng_polar_noalloc(_p(out), 0, 0.0, 1.0, 3, 12345, 0, 0, _p(nxt), None, _p(status), stream) == _lib.OK
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert int(nxt.item()) == 12345


def test_noalloc_refuses_n_beyond_its_scratch():
    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = torch.empty(16, dtype=torch.float32, device="cuda")
    # n larger than the fixed array serves: rejected before anything is enqueued
    rc = lib.nrng_polar_noalloc(_p(out), (1 << 28) + 1, 0.0, 1.0, 1, 0, 0, 0, None, None, None, stream)
    assert rc == _lib.ERR_WORKSPACE
    assert "workspace" in lib.nrng_status_string(rc).decode()
