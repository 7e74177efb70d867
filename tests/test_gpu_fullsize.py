"""Parity at the full single-stream size N = 2^28 in the launch configuration
the benchmark times: B1 on sampled outputs the oracle computes one by one;
Polar with the accept order checked over every candidate (the oracle's
accept bits up to the last consumed candidate) and values at sampled pairs
from their candidate indices; the precision sweep (mu 1.5, sigma 0.25) over
{B1, P} x {accurate, fast} x {f32, bf16, f16} on sampled outputs, and on the
tails (every output the oracle's uniforms put at |z| >= 4)."""
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


@pytest.fixture(scope="module")
def tail_points(polar_full):
    """Outputs of the 2^28 streams (key 0x5EED0001, counter 0) that lie in the
    tails, found from the oracle's Philox words chunk by chunk: B1 pairs with
    u >= 1 - 2^-12 (r >= 4.08), and the Polar pairs with |z| >= 4 on either
    coordinate (with their candidate indices)."""
    chunk = 1 << 22
    b1_idx = []
    for b0 in range(0, N // 4, chunk):
        w = oracle.philox_blocks(min(chunk, N // 4 - b0), W.KEY_MAIN, b0)
        for p in (0, 1):
            hit = np.flatnonzero((w[:, 2 * p] >> 8) >= (1 << 24) - (1 << 12))
            b = (b0 + hit).astype(np.int64)
            b1_idx += [4 * b + 2 * p, 4 * b + 2 * p + 1]
    b1_idx = np.sort(np.concatenate(b1_idx))
    _, cand, _ = polar_full
    ncand = int(cand[-1]) + 1
    tail_c = []
    for b0 in range(0, (ncand + 1) // 2, chunk):
        w = oracle.philox_blocks(min(chunk, (ncand + 1) // 2 - b0), W.KEY_MAIN, b0).astype(np.int64)
        kx = (w[:, [0, 2]] >> 8).ravel() - (1 << 23)
        ky = (w[:, [1, 3]] >> 8).ravel() - (1 << 23)
        S = kx * kx + ky * ky
        ok = (S > 0) & (S < (1 << 46))
        s_ = np.where(ok, S, 1).astype(np.float64) * 2.0 ** -46
        g = np.sqrt(-2.0 * np.log(s_) / s_) * 2.0 ** -23
        big = ok & (np.maximum(np.abs(kx), np.abs(ky)) * g >= 4.0)
        tail_c.append(2 * b0 + np.flatnonzero(big))
    tail_c = np.concatenate(tail_c)
    tail_c = tail_c[tail_c < ncand]
    pairs = np.searchsorted(cand, tail_c)
    assert np.array_equal(cand[pairs], tail_c)
    return b1_idx, pairs, tail_c


@pytest.mark.parametrize("method", ["b1", "polar"])
@pytest.mark.parametrize("mode", ["accurate", "fast"])
def test_tails_full_size(method, mode, tail_points):
    """The tails of the precision sweep (mu 1.5, sigma 0.25, fp32, N = 2^28)
    against the oracle: the |z|-binned errors up to |z| = 8."""
    mu, sigma = W.SWEEP_MU, W.SWEEP_SIGMA
    b1_idx, pairs, tail_c = tail_points
    out = torch.empty(N, dtype=torch.float32, device="cuda")
    if method == "b1":
        nr.nrng_boxmuller(out, mu, sigma, W.KEY_MAIN, 0, mode)
        sync()
        idx = b1_idx
        ref = oracle.boxmuller_at(idx, mu, sigma, W.KEY_MAIN, 0)
        assert np.abs((ref - mu) / sigma).max() >= 5.0
    else:
        ws = nr.polar_workspace(N)
        nr.nrng_polar(out, mu, sigma, W.KEY_MAIN, 0, ws, mode)
        assert nr.nrng_get_status(ws) == 0
        idx = np.stack([2 * pairs, 2 * pairs + 1], axis=1).ravel()
        ref = oracle.polar_at(tail_c, mu, sigma, W.KEY_MAIN, 0).ravel()
        assert np.abs((ref - mu) / sigma).max() >= 5.0
    got = out[torch.from_numpy(idx).cuda()]
    assert_close(got, ref, mu, sigma, mode, f"tails {method} {mode}")
    record_error_table(f"{method} {mode} float32 tails", got, ref, mu, sigma, N)

