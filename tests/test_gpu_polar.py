"""GPU parity of Algorithm P (Sec. 2) with order-preserving compaction
against the FP64 oracle, through the C ABI: the candidate index of every
output pair and next_counter bit-exact, values within tolerance, for every
mode x dtype, odd and tiny n, unaligned outputs; continuation; normality."""
import numpy as np
import pytest
import torch

import oracle
import paper_1004_3105_gb300 as nr
from gpu_helpers import assert_canary, assert_close, canary_tensor, sync
from paper_1004_3105_gb300 import workloads as W
from stats import check_standard_normal_moments, ks_critical, ks_distance, normal_cdf

pytestmark = pytest.mark.gpu
DTYPES = [torch.float32, torch.bfloat16, torch.float16]


def run_polar(n, mu, sigma, key, counter, mode="accurate", dtype=torch.float32, offset=0):
    whole, out = canary_tensor(n, dtype, offset=offset)
    ws = nr.polar_workspace(n)
    nxt = torch.zeros(1, dtype=torch.int64, device="cuda")
    cand = torch.full(((n + 1) // 2,), -1, dtype=torch.int64, device="cuda")
    nr.nrng_polar(out, mu, sigma, key, counter, ws, mode, next_counter=nxt, pair_candidate=cand)
    status = nr.nrng_get_status(ws)
    assert status == 0, nr._lib.STATUS[status]
    assert_canary(whole, offset, n)
    return out, cand.cpu().numpy(), int(nxt.item()) & 0xFFFFFFFFFFFFFFFF


@pytest.mark.parametrize("n", [1, 2, 3, 5, 4095, 4096, 4097, 65537, 1 << 22])
def test_polar_accurate_f32(n):
    out, cand, nxt = run_polar(n, 0.0, 1.0, W.KEY_MAIN, 0)
    ref, rcand, rnxt, _ = oracle.polar(n, 0.0, 1.0, W.KEY_MAIN, 0)
    assert np.array_equal(cand, rcand), "accept order"
    assert nxt == rnxt
    assert_close(out, ref, 0.0, 1.0, "accurate", f"polar n={n}")


@pytest.mark.parametrize("mode", ["accurate", "fast"])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n,offset", [(100003, 0), (4097, 1)])
def test_polar_modes_dtypes(mode, dtype, n, offset):
    mu, sigma = W.SWEEP_MU, W.SWEEP_SIGMA
    out, cand, nxt = run_polar(n, mu, sigma, W.KEY_MAIN, 3, mode, dtype, offset)
    ref, rcand, rnxt, _ = oracle.polar(n, mu, sigma, W.KEY_MAIN, 3)
    assert np.array_equal(cand, rcand)
    assert nxt == rnxt
    assert_close(out, ref, mu, sigma, mode, f"polar {mode} {dtype}")


def test_polar_config_c2_side_by_side():
    """Polar N = 2^26 fp32 (mu 0, sigma 1, key 0x5EED0001, counter 0) next to B1."""
    n = W.N_PARITY_POLAR
    out, cand, nxt = run_polar(n, 0.0, 1.0, W.KEY_MAIN, 0)
    ref, rcand, rnxt, _ = oracle.polar(n, 0.0, 1.0, W.KEY_MAIN, 0)
    assert np.array_equal(cand, rcand)
    assert nxt == rnxt
    assert_close(out, ref, 0.0, 1.0, "accurate", "polar C2")
    b1 = torch.empty(n, dtype=torch.float32, device="cuda")
    nr.nrng_boxmuller(b1, 0.0, 1.0, W.KEY_MAIN, 0)
    sync()
    idx = W.sample_indices(n, 1 << 20)
    assert_close(b1[torch.from_numpy(idx).cuda()], oracle.boxmuller_at(idx, 0.0, 1.0, W.KEY_MAIN, 0),
                 0.0, 1.0, "accurate", "B1 C2")


def test_polar_continuation():
    """next_counter continues the stream: generating n1 then n2 from it gives
    the oracle's stream restarted at that counter."""
    n1, n2 = 10001, 7000
    out1, _, nxt = run_polar(n1, 0.0, 1.0, 77, 5)
    out2, _, _ = run_polar(n2, 0.0, 1.0, 77, nxt)
    _, _, rnxt, _ = oracle.polar(n1, 0.0, 1.0, 77, 5)
    assert nxt == rnxt
    ref2, _, _, _ = oracle.polar(n2, 0.0, 1.0, 77, rnxt)
    assert_close(out2, ref2, 0.0, 1.0, "accurate", "continuation")


def test_polar_zero_n_sets_next_counter():
    ws = nr.polar_workspace(1)
    nxt = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = torch.empty(0, dtype=torch.float32, device="cuda")
    nr.nrng_polar(out, 0.0, 1.0, 1, 12345, ws, next_counter=nxt)
    sync()
    assert int(nxt.item()) == 12345


@pytest.mark.parametrize("mode", ["accurate", "fast"])
def test_polar_normality_and_acceptance(mode):
    n = 1_000_000
    out, cand, nxt = run_polar(n, 0.0, 1.0, 31337, 0, mode)
    z = out.cpu().numpy().astype(np.float64)
    check_standard_normal_moments(z)
    assert ks_distance(z, normal_cdf) < ks_critical(n)
    # candidates examined per pair -> 4/pi
    c_last = cand[-1] + 1
    p = oracle.lattice_accept_count() / 2.0 ** 48
    k = cand.size
    assert abs(k - c_last * p) < 5 * np.sqrt(c_last * p * (1 - p))


def test_polar_repeat_is_deterministic():
    n = 1 << 21
    a, ca, na = run_polar(n, 0.0, 1.0, 9, 0, "fast")
    b, cb, nb = run_polar(n, 0.0, 1.0, 9, 0, "fast")
    assert torch.equal(a, b) and np.array_equal(ca, cb) and na == nb


@pytest.mark.parametrize("mode", ["accurate", "fast"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("n,offset", [(1, 0), (4097, 1), (100003, 0), (1 << 22, 0)])
def test_polar_twopass_equals_single_pass(mode, dtype, n, offset):
    """The count/scan/write form gives nrng_polar's outputs bit for bit."""
    mu, sigma = W.SWEEP_MU, W.SWEEP_SIGMA
    one, cand1, nxt1 = run_polar(n, mu, sigma, W.KEY_MAIN, 9, mode, dtype, offset)
    whole, out = canary_tensor(n, dtype, offset=offset)
    ws = torch.empty(nr.nrng_polar_twopass_workspace_size(n), dtype=torch.uint8, device="cuda")
    nxt = torch.zeros(1, dtype=torch.int64, device="cuda")
    cand = torch.full(((n + 1) // 2,), -1, dtype=torch.int64, device="cuda")
    nr.nrng_polar_twopass(out, mu, sigma, W.KEY_MAIN, 9, ws, mode, next_counter=nxt, pair_candidate=cand)
    assert nr.nrng_get_status(ws) == 0
    assert_canary(whole, offset, n)
    assert torch.equal(out, one)
    assert np.array_equal(cand.cpu().numpy(), cand1)
    assert int(nxt.item()) == nxt1


def test_polar_twopass_oracle_and_budget():
    n = 300001
    ws = torch.empty(nr.nrng_polar_twopass_workspace_size(n), dtype=torch.uint8, device="cuda")
    out = torch.empty(n, device="cuda")
    nr.nrng_polar_twopass(out, 0.0, 1.0, 5, 0, ws, "accurate")
    assert nr.nrng_get_status(ws) == 0
    assert_close(out, oracle.polar(n, 0.0, 1.0, 5, 0)[0], 0.0, 1.0, "accurate", "twopass")
