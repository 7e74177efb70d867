"""Parity at the full single-stream size N = 2^28 in the launch configuration
the benchmark times: B1 on sampled outputs the oracle computes one by one;
Polar with the accept order checked over every candidate (the oracle's
accept bits up to the last consumed candidate) and values at sampled pairs
from their candidate indices; the precision sweep (mu 1.5, sigma 0.25) over
{B1, P} x {accurate, fast} x {f32, bf16, f16} on sampled outputs."""
import numpy as np
import pytest
import torch

import oracle
import paper_1004_3105_gb300 as nr
from gpu_helpers import assert_close, record_error_table, sync
from paper_1004_3105_gb300 import workloads as W

pytestmark = pytest.mark.gpu
N = W.N_FULL


@pytest.fixture(scope="module")
def polar_full():
    out = torch.empty(N, dtype=torch.float32, device="cuda")
    ws = nr.polar_workspace(N)
    cand = torch.empty(N // 2, dtype=torch.int64, device="cuda")
    nxt = torch.zeros(1, dtype=torch.int64, device="cuda")
    nr.nrng_polar(out, 0.0, 1.0, W.KEY_MAIN, 0, ws, "accurate", next_counter=nxt, pair_candidate=cand)
    assert nr.nrng_get_status(ws) == 0
    c = cand.cpu().numpy()
    del cand
    return out, c, int(nxt.item())


def test_b1_full_sampled():
    out = torch.empty(N, dtype=torch.float32, device="cuda")
    nr.nrng_boxmuller(out, 0.0, 1.0, W.KEY_MAIN, 0, "accurate")
    sync()
    idx = W.sample_indices(N, 1 << 19)
    assert_close(out[torch.from_numpy(idx).cuda()], oracle.boxmuller_at(idx, 0.0, 1.0, W.KEY_MAIN, 0),
                 0.0, 1.0, "accurate", "B1 2^28")


def test_polar_full_accept_order(polar_full):
    out, cand, nxt = polar_full
    ncand = int(cand[-1]) + 1
    acc, _, _ = oracle.polar_candidates(ncand, W.KEY_MAIN, 0, coords=False)
    want = np.flatnonzero(acc)
    assert want.size == N // 2
    assert np.array_equal(cand, want)
    assert nxt == cand[-1] // 2 + 1


def test_polar_full_sampled_values(polar_full):
    out, cand, _ = polar_full
    pairs = W.sample_indices(N // 2, 1 << 18)
    ref = oracle.polar_at(cand[pairs], 0.0, 1.0, W.KEY_MAIN, 0)
    got_idx = torch.from_numpy(np.stack([2 * pairs, 2 * pairs + 1], axis=1).ravel()).cuda()
    assert_close(out[got_idx], ref.ravel(), 0.0, 1.0, "accurate", "polar 2^28")


@pytest.mark.parametrize("method", ["b1", "polar"])
@pytest.mark.parametrize("mode", ["accurate", "fast"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
def test_precision_sweep_sampled(method, mode, dtype, polar_full):
    mu, sigma = W.SWEEP_MU, W.SWEEP_SIGMA
    out = torch.empty(N, dtype=dtype, device="cuda")
    if method == "b1":
        nr.nrng_boxmuller(out, mu, sigma, W.KEY_MAIN, 0, mode)
        sync()
        idx = W.sample_indices(N, 1 << 18)
        ref = oracle.boxmuller_at(idx, mu, sigma, W.KEY_MAIN, 0)
    else:
        ws = nr.polar_workspace(N)
        nr.nrng_polar(out, mu, sigma, W.KEY_MAIN, 0, ws, mode)
        assert nr.nrng_get_status(ws) == 0
        _, cand, _ = polar_full      # the accept order does not depend on mode, dtype, mu or sigma
        pairs = W.sample_indices(N // 2, 1 << 17)
        ref = oracle.polar_at(cand[pairs], mu, sigma, W.KEY_MAIN, 0).ravel()
        idx = np.stack([2 * pairs, 2 * pairs + 1], axis=1).ravel()
    got = out[torch.from_numpy(idx).cuda()]
    assert_close(got, ref, mu, sigma, mode, f"sweep {method} {mode} {dtype}")
    record_error_table(f"{method} {mode} {str(dtype).replace('torch.', '')}", got, ref, mu, sigma, N)
