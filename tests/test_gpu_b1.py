"""GPU parity of uniforms and Algorithm B1 (Sec. 2) against the FP64 oracle,
through the C ABI: bit-exact uniforms; B1 values within the stated tolerance
for every mode x dtype, ragged tails, unaligned outputs and counter carries;
normality of the GPU output."""
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


@pytest.mark.parametrize("n", [0, 1, 3, 4, 5, 4095, 4097, (1 << 20) + 3])
@pytest.mark.parametrize("offset", [0, 1])
def test_uniform_bit_exact(n, offset):
    whole, out = canary_tensor(n, torch.float32, offset=offset)
    nr.nrng_uniform(out, W.KEY_MAIN, 7)
    sync()
    ref = oracle.uniform(n, W.KEY_MAIN, 7).astype(np.float32)
    assert np.array_equal(out.cpu().numpy(), ref)
    assert_canary(whole, offset, n)


def test_uniform_counter_carry_and_high_key():
    key, counter = 0x123456789ABCDEF0, (1 << 32) - 3
    out = torch.empty(64, dtype=torch.float32, device="cuda")
    nr.nrng_uniform(out, key, counter)
    sync()
    assert np.array_equal(out.cpu().numpy(), oracle.uniform(64, key, counter).astype(np.float32))


def test_boxmuller_config_c1():
    """B1, N = 2^20, mu 0, sigma 1, key 0x5EED0001, counter 0, accurate, fp32."""
    n = W.N_PARITY_B1
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    nr.nrng_boxmuller(out, 0.0, 1.0, W.KEY_MAIN, W.COUNTER0, "accurate")
    sync()
    ref = oracle.boxmuller(n, 0.0, 1.0, W.KEY_MAIN, W.COUNTER0)
    worst = assert_close(out, ref, 0.0, 1.0, "accurate", "B1 C1")
    assert worst < 4e-6


@pytest.mark.parametrize("mode", ["accurate", "fast"])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n,offset", [(65539, 0), (4097, 1), (5, 3), (1, 0)])
def test_boxmuller_modes_dtypes_tails(mode, dtype, n, offset):
    mu, sigma = W.SWEEP_MU, W.SWEEP_SIGMA
    whole, out = canary_tensor(n, dtype, offset=offset)
    nr.nrng_boxmuller(out, mu, sigma, W.KEY_MAIN, 11, mode)
    sync()
    ref = oracle.boxmuller(n, mu, sigma, W.KEY_MAIN, 11)
    assert_close(out, ref, mu, sigma, mode, f"B1 {mode} {dtype} n={n}")
    assert_canary(whole, offset, n)


def test_boxmuller_sigma_zero_and_counter_carry():
    out = torch.empty(1001, dtype=torch.float32, device="cuda")
    nr.nrng_boxmuller(out, 2.5, 0.0, W.KEY_MAIN, 0)
    sync()
    assert torch.all(out == 2.5)
    counter = (1 << 32) - 17
    nr.nrng_boxmuller(out, -1.0, 3.0, 99, counter, "fast")
    sync()
    assert_close(out, oracle.boxmuller(1001, -1.0, 3.0, 99, counter), -1.0, 3.0, "fast", "carry")


@pytest.mark.parametrize("mode", ["accurate", "fast"])
def test_boxmuller_normality(mode):
    n = 1_000_000
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    nr.nrng_boxmuller(out, 0.0, 1.0, 2024, 0, mode)
    sync()
    z = out.cpu().numpy().astype(np.float64)
    check_standard_normal_moments(z)
    assert ks_distance(z, normal_cdf) < ks_critical(n)


def test_boxmuller_stream_continuation():
    """Two calls with counter + ceil(n/4) concatenate into one stream."""
    a = torch.empty(4096, dtype=torch.float32, device="cuda")
    b = torch.empty(2048, dtype=torch.float32, device="cuda")
    c = torch.empty(2048, dtype=torch.float32, device="cuda")
    nr.nrng_boxmuller(a, 0.0, 1.0, 5, 100)
    nr.nrng_boxmuller(b, 0.0, 1.0, 5, 100)
    nr.nrng_boxmuller(c, 0.0, 1.0, 5, 100 + 512)
    sync()
    assert torch.equal(a, torch.cat([b, c]))


@pytest.mark.parametrize("nblocks,counter", [(1, 0), (100003, 5), (1 << 20, (7 << 32) + 11)])
def test_philox_ceiling_draws_every_block(nblocks, counter):
    # the measurement kernel draws exactly the blocks [counter, counter + nblocks):
    # the xor of all their words equals the oracle's
    acc = torch.zeros(1, dtype=torch.int32, device="cuda")
    nr.nrng_philox_ceiling(acc, nblocks, W.KEY_MAIN, counter)
    sync()
    want = int(np.bitwise_xor.reduce(oracle.philox_blocks(nblocks, W.KEY_MAIN, counter).astype(np.uint32).ravel()))
    assert (int(acc.item()) & 0xFFFFFFFF) == want
