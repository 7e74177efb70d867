"""GPU parity of the batched launch (every configuration, graph replay,
autotuner, device-side descriptor errors) and of the reparameterised sample
and its autograd backward, against the FP64 oracle through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import paper_1004_3105_gb300 as nr
from gpu_helpers import assert_close, sync
from paper_1004_3105_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def make_batch(k, len_lo, len_hi, methods, align, dtype=torch.float32, seed=W.BATCH_SEED):
    wl = W.batched_workload(k=k, seed=seed, methods=methods, len_lo=len_lo, len_hi=len_hi, align=align)
    desc = nr.stream_descriptors(wl.offset, wl.n, wl.mu, wl.sigma, wl.key, wl.counter, wl.method)
    pad = 64
    out = torch.full((wl.total + pad,), -12345.0, dtype=dtype, device="cuda")
    ws = torch.empty(max(nr.nrng_batched_workspace_size(desc), 256), dtype=torch.uint8, device="cuda")
    return wl, desc, nr.descriptors_to_device(desc), out, ws


def check_batch(wl, out, mode, what):
    ref = oracle.batched(wl.total, wl.as_dict())
    got = out[:wl.total]
    for j in range(len(wl.n)):
        o, n = int(wl.offset[j]), int(wl.n[j])
        assert_close(got[o:o + n], ref[o:o + n], float(wl.mu[j]), float(wl.sigma[j]), mode,
                     f"{what} stream {j} (method {wl.method[j]}, n {n})")
    sentinel = float(torch.tensor(-12345.0, dtype=out.dtype).float())
    tail = out[wl.total:].float().cpu().numpy()
    assert np.all(tail == sentinel)
    # gaps between aligned streams stay untouched
    mask = np.ones(wl.total, dtype=bool)
    for j in range(len(wl.n)):
        mask[int(wl.offset[j]):int(wl.offset[j]) + int(wl.n[j])] = False
    if mask.any():
        assert np.all(got.float().cpu().numpy()[mask] == sentinel)


@pytest.mark.parametrize("config", range(7))
def test_batched_every_config(config):
    wl, desc, d_desc, out, ws = make_batch(64, 1, 20000, "mixed", align=1)
    nr.nrng_batched_set_config(torch.float32, "accurate", config)
    try:
        nr.nrng_batched(out, d_desc, len(desc), ws, "accurate")
        assert nr.nrng_get_status(ws) == 0
    finally:
        nr.nrng_batched_set_config(torch.float32, "accurate", -1)
    check_batch(wl, out, "accurate", f"config {config}")


@pytest.mark.parametrize("config", range(6))
def test_batched_long_polar_streams_every_config(config):
    """Few long Polar streams: hundreds of tiles of one stream in flight at
    once, so tiles are taken after their stream completed (the skip path) and
    look-back windows slide past 32 predecessors."""
    wl, desc, d_desc, out, ws = make_batch(6, 3e5, 1e6, "polar", align=2, seed=3)
    nr.nrng_batched_set_config(torch.float32, "fast", config)
    try:
        for _ in range(3):
            nr.nrng_batched(out, d_desc, len(desc), ws, "fast")
            assert nr.nrng_get_status(ws) == 0
    finally:
        nr.nrng_batched_set_config(torch.float32, "fast", -1)
    check_batch(wl, out, "fast", f"long polar config {config}")


@pytest.mark.parametrize("mode", ["accurate", "fast"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
@pytest.mark.parametrize("methods,align", [("b1", 4), ("polar", 2), ("mixed", 1)])
def test_batched_modes_dtypes(mode, dtype, methods, align):
    wl, desc, d_desc, out, ws = make_batch(48, 1, 30000, methods, align, dtype)
    nr.nrng_batched(out, d_desc, len(desc), ws, mode)
    assert nr.nrng_get_status(ws) == 0
    check_batch(wl, out, mode, f"{methods} {mode} {dtype}")


def test_batched_full_workload_sampled():
    """4096 streams, lengths log-uniform in [1e2, 1e6] (seed 7), mixed B1/P,
    one persistent launch; a sample of 48 whole streams checked."""
    wl, desc, d_desc, out, ws = make_batch(W.BATCH_STREAMS, W.BATCH_LEN_LO, W.BATCH_LEN_HI, "mixed", align=4)
    nr.nrng_batched(out, d_desc, len(desc), ws, "accurate")
    assert nr.nrng_get_status(ws) == 0
    rng = np.random.Generator(np.random.PCG64(1))
    pick = np.unique(np.concatenate([rng.choice(len(desc), 46, replace=False), [0, len(desc) - 1]]))
    for j in pick:
        o, n = int(wl.offset[j]), int(wl.n[j])
        mu, sg, key = float(wl.mu[j]), float(wl.sigma[j]), int(wl.key[j])
        ref = oracle.boxmuller(n, mu, sg, key, 0) if wl.method[j] == 0 else oracle.polar(n, mu, sg, key, 0)[0]
        assert_close(out[o:o + n], ref, mu, sg, "accurate", f"stream {j}")


def test_batched_full_workload_every_short_stream():
    """The same 4096-stream launch in every tile configuration; every stream
    of at most 2e4 normals (about a third of them: one or two primary tiles,
    the rest from the overflow item) checked whole."""
    wl, desc, d_desc, out, ws = make_batch(W.BATCH_STREAMS, W.BATCH_LEN_LO, W.BATCH_LEN_HI, "mixed", align=4)
    short = np.flatnonzero(wl.n <= 20000)
    assert short.size > 1000
    refs = {}
    for j in short:
        n, mu, sg, key = int(wl.n[j]), float(wl.mu[j]), float(wl.sigma[j]), int(wl.key[j])
        refs[j] = oracle.boxmuller(n, mu, sg, key, 0) if wl.method[j] == 0 else oracle.polar(n, mu, sg, key, 0)[0]
    for config in range(nr.nrng_batched_config_count()):
        out.fill_(0.0)
        nr.nrng_batched_set_config(torch.float32, "accurate", config)
        try:
            nr.nrng_batched(out, d_desc, len(desc), ws, "accurate")
            assert nr.nrng_get_status(ws) == 0
        finally:
            nr.nrng_batched_set_config(torch.float32, "accurate", -1)
        got = out.cpu()
        for j in short:
            o, n = int(wl.offset[j]), int(wl.n[j])
            assert_close(got[o:o + n], refs[j], float(wl.mu[j]), float(wl.sigma[j]), "accurate",
                         f"config {config} stream {j}")


def test_batched_graph_and_autotune_agree():
    wl, desc, d_desc, out, ws = make_batch(96, 10, 50000, "mixed", align=1)
    nr.nrng_batched(out, d_desc, len(desc), ws, "fast")
    sync()
    direct = out.clone()
    out.fill_(0.0)
    g = nr.BatchedGraph(out, d_desc, len(desc), ws, "fast")
    g.launch()
    g.launch()
    sync()
    assert torch.equal(out[:wl.total], direct[:wl.total])
    g.close()
    cfg, ms = nr.nrng_batched_autotune(out, d_desc, len(desc), ws, "fast", reps=2)
    assert 0 <= cfg < nr.nrng_batched_config_count() and ms > 0
    assert nr.nrng_batched_get_config(torch.float32, "fast") == cfg
    out.fill_(0.0)
    nr.nrng_batched(out, d_desc, len(desc), ws, "fast")
    sync()
    nr.nrng_batched_set_config(torch.float32, "fast", -1)
    # the outputs do not depend on the tile shape
    assert torch.equal(out[:wl.total], direct[:wl.total])


def test_batched_autotune_cache(tmp_path, monkeypatch):
    """NRNG_AUTOTUNE_CACHE: the first tuning of a workload appends one line;
    the same workload shape (other keys and parameters) reuses it without
    timing; a different shape is tuned and appended."""
    cache = tmp_path / "autotune.jsonl"
    monkeypatch.setenv("NRNG_AUTOTUNE_CACHE", str(cache))
    wl, desc, d_desc, out, ws = make_batch(40, 10, 20000, "mixed", align=1)
    cfg, ms = nr.nrng_batched_autotune(out, d_desc, len(desc), ws, "accurate", reps=1)
    assert len(cache.read_text().splitlines()) == 1
    nr.nrng_batched_set_config(torch.float32, "accurate", -1)
    desc2 = desc.copy()
    desc2["key"] += 1000
    desc2["mu"] = 0.5
    cfg2, ms2 = nr.nrng_batched_autotune(out, nr.descriptors_to_device(desc2), len(desc2), ws, "accurate", reps=1)
    assert cfg2 == cfg and ms2 == pytest.approx(ms, abs=2e-6)
    assert len(cache.read_text().splitlines()) == 1
    assert nr.nrng_batched_get_config(torch.float32, "accurate") == cfg
    desc3 = desc.copy()
    desc3["n"][0] += 1
    desc3["offset"] = np.concatenate([[0], np.cumsum(desc3["n"])[:-1]])
    ws3 = torch.empty(max(nr.nrng_batched_workspace_size(desc3), 256), dtype=torch.uint8, device="cuda")
    out3 = torch.empty(int(desc3["offset"][-1] + desc3["n"][-1]) + 64, device="cuda")
    nr.nrng_batched_autotune(out3, nr.descriptors_to_device(desc3), len(desc3), ws3, "accurate", reps=1)
    assert len(cache.read_text().splitlines()) == 2
    nr.nrng_batched_set_config(torch.float32, "accurate", -1)


def test_batched_device_descriptor_errors():
    wl, desc, d_desc, out, ws = make_batch(8, 10, 1000, "mixed", align=1)
    bad = desc.copy()
    bad["sigma"][3] = -1.0
    d_bad = nr.descriptors_to_device(bad)
    before = out.clone()
    nr.nrng_batched(out, d_bad, len(bad), ws, "accurate")
    assert nr.nrng_get_status(ws) == nr._lib.ERR_INVALID_VALUE
    assert torch.equal(out, before)          # nothing written
    # a workspace large enough for the tables but not for the tile words
    # (the header and per-stream tables of 8 streams take 512 bytes; the 4
    # Polar streams need >= 4 words)
    small = torch.empty(520, dtype=torch.uint8, device="cuda")
    nr.nrng_batched(out, d_desc, len(desc), small, "accurate")
    assert nr.nrng_get_status(small) == nr._lib.ERR_WORKSPACE
    assert torch.equal(out, before)
    # and the context is fine afterwards
    nr.nrng_batched(out, d_desc, len(desc), ws, "accurate")
    assert nr.nrng_get_status(ws) == 0
    check_batch(wl, out, "accurate", "after errors")


def test_batched_many_streams_setup_lookback():
    """20,000 short streams: the setup places them with a block scan per 256
    streams and a look-back across 79 CTAs, more than its 32-wide window
    covers, so a CTA whose nearer predecessors have not yet published their
    prefixes walks back over several windows.  Every stream must match the
    oracle."""
    wl, desc, d_desc, out, ws = make_batch(20000, 1, 64, "mixed", align=1)
    nr.nrng_batched(out, d_desc, len(desc), ws, "accurate")
    assert nr.nrng_get_status(ws) == 0
    check_batch(wl, out, "accurate", "20000 streams")


def test_batched_short_stream_tile0_second_draw():
    """A Polar stream shorter than a tile draws, in its tile 0, only the warps
    that reach into the candidates it is expected to need (nitems / (pi/4)),
    and the other warps only when those fall short.  Streams whose expected
    need sits just below a warp boundary (1152 candidates a warp in the
    default 128 x 18 configuration) are picked with the oracle's accept bits
    so that both cases occur: some fall short and take the second draw, some
    do not.  Every stream must match the oracle and, bit for bit, the
    single-stream kernel."""
    per_warp = 18 * 64
    picked, short, enough = [], 0, 0
    for key in range(1, 2000):
        if short >= 6 and enough >= 6:
            break
        for nitems in (900, 904, 1808, 1809):
            limit = int(np.float32(nitems) * np.float32(1.2732395))
            warps = -(-limit // per_warp)
            acc, _, _ = oracle.polar_candidates(warps * per_warp, key, 0, coords=False)
            falls_short = int(acc.sum()) < nitems
            if (falls_short and short < 6) or (not falls_short and enough < 6):
                picked.append((key, 2 * nitems))
                short += falls_short
                enough += not falls_short
    assert short >= 6 and enough >= 6
    n = np.array([m for _, m in picked], dtype=np.int64)
    offset = np.concatenate([[0], np.cumsum(n)[:-1]]).astype(np.int64)
    k = len(n)
    mu, sigma = np.full(k, 0.5, np.float32), np.full(k, 1.5, np.float32)
    key = np.array([q for q, _ in picked], dtype=np.uint64)
    desc = nr.stream_descriptors(offset, n, mu, sigma, key, np.zeros(k, np.uint64), np.ones(k, np.int32))
    total = int(n.sum())
    out = torch.full((total,), -12345.0, dtype=torch.float32, device="cuda")
    ws = torch.empty(nr.nrng_batched_workspace_size(desc), dtype=torch.uint8, device="cuda")
    nr.nrng_batched_set_config(torch.float32, "accurate", 0)
    nr.nrng_batched(out, nr.descriptors_to_device(desc), k, ws, "accurate")
    assert nr.nrng_get_status(ws) == 0
    got = out.cpu()
    for j in range(k):
        o, m = int(offset[j]), int(n[j])
        ref, _, _, _ = oracle.polar(m, 0.5, 1.5, int(key[j]), 0)
        assert_close(got[o:o + m].cuda(), ref, 0.5, 1.5, "accurate", f"short stream {j} (key {int(key[j])}, n {m})")
        one = torch.empty(m, dtype=torch.float32, device="cuda")
        wsp = nr.polar_workspace(m)
        nr.nrng_polar(one, 0.5, 1.5, int(key[j]), 0, wsp, "accurate")
        assert torch.equal(one.cpu(), got[o:o + m]), f"short stream {j}: batched differs from nrng_polar"


# ------------------------------------------------------------------ reparam
@pytest.mark.parametrize("mode", ["accurate", "fast"])
def test_reparam_config_c5(mode):
    wl = W.reparam_workload()
    shape = W.REPARAM_SHAPE
    n = int(np.prod(shape))
    mu = torch.from_numpy(wl.mu).cuda()
    sigma = torch.from_numpy(wl.sigma).cuda()
    x = torch.empty(shape, dtype=torch.float32, device="cuda")
    nr.nrng_reparam_fwd(x, mu, sigma, W.KEY_REPARAM, 0, mode)
    sync()
    xr = oracle.reparam_fwd(wl.mu, wl.sigma, n, 1, W.KEY_REPARAM, 0)
    z = oracle.boxmuller(n, 0.0, 1.0, W.KEY_REPARAM, 0)
    got = x.cpu().numpy().ravel().astype(np.float64)
    # x = mu + sigma z: bound in z units scaled by each element's sigma
    s64 = wl.sigma.ravel().astype(np.float64)
    from gpu_helpers import TOL, ulp_fmt
    bnd = TOL[mode] * s64 * np.maximum(1, np.abs(z)) + ulp_fmt(xr, torch.float32)
    assert np.all(np.abs(got - xr) <= bnd)
    # backward of loss = sum(w x^2): g = 2 w x
    g = (2.0 * torch.from_numpy(wl.w).cuda() * x).contiguous()
    dmu = torch.empty_like(mu)
    dsig = torch.empty_like(sigma)
    nr.nrng_reparam_bwd(dmu, dsig, g, W.KEY_REPARAM, 0, mode)
    sync()
    gh = g.cpu().numpy().ravel()
    rdmu, rdsig = oracle.reparam_bwd(gh, n, 1, W.KEY_REPARAM, 0)
    assert np.array_equal(dmu.cpu().numpy().ravel(), gh)
    gz = np.abs(gh.astype(np.float64))
    assert np.all(np.abs(dsig.cpu().numpy().ravel() - rdsig) <= TOL[mode] * gz * np.maximum(1, np.abs(z)) +
                  ulp_fmt(rdsig, torch.float32))


@pytest.mark.parametrize("pshape", [(1,), (8192,), (1024, 1), (1024, 8192)])
def test_reparam_autograd_broadcast(pshape):
    shape = (1024, 8192) if pshape != (1,) else (256, 1024)
    n = int(np.prod(shape))
    rng = np.random.Generator(np.random.PCG64(2))
    mu_h = rng.standard_normal(size=pshape).astype(np.float32)
    sg_h = rng.uniform(0.1, 2.0, size=pshape).astype(np.float32)
    w_h = rng.uniform(-1, 1, size=shape).astype(np.float32)
    mu = torch.from_numpy(mu_h).cuda().requires_grad_(True)
    sg = torch.from_numpy(sg_h).cuda().requires_grad_(True)
    w = torch.from_numpy(w_h).cuda()
    x = nr.Reparam.apply(mu, sg, shape, W.KEY_REPARAM, 0, "accurate")
    loss = (w * x * x).sum()
    loss.backward()
    m, inner = nr.broadcast_layout(pshape, shape)
    g = (2.0 * w * x).detach().cpu().numpy().ravel()
    rdmu, rdsig = oracle.reparam_bwd(g, m, inner, W.KEY_REPARAM, 0)
    # sums of n/m float terms: float32 accumulation in any order stays within
    # (count * 2^-24 + 4e-6) of the sum of absolute terms
    z = oracle.boxmuller(n, 0.0, 1.0, W.KEY_REPARAM, 0)
    absg = np.abs(g.astype(np.float64))
    idx = (np.arange(n) // inner) % m
    abs_gz = np.bincount(idx, weights=absg * np.maximum(1, np.abs(z)), minlength=m)
    abs_g = np.bincount(idx, weights=absg, minlength=m)
    cnt = n // m
    slack = cnt * 2.0 ** -24 + 4e-6
    assert np.all(np.abs(mu.grad.cpu().numpy().ravel() - rdmu) <= slack * abs_g + 1e-6)
    assert np.all(np.abs(sg.grad.cpu().numpy().ravel() - rdsig) <= slack * abs_gz + 1e-6)


def test_reparam_recompute_equals_stream():
    """z seen by forward (mu 0, sigma 1) and by backward (g 1 -> dsigma = z) is
    bitwise the nrng_boxmuller stream of the same key and counter."""
    n = (1 << 20) + 6
    for mode in ("accurate", "fast"):
        zero = torch.zeros(n, device="cuda")
        one = torch.ones(n, device="cuda")
        x = torch.empty(n, device="cuda")
        nr.nrng_reparam_fwd(x, zero, one, 42, 9, mode)
        dsig = torch.empty(n, device="cuda")
        nr.nrng_reparam_bwd(None, dsig, one, 42, 9, mode)
        ref = torch.empty(n, device="cuda")
        nr.nrng_boxmuller(ref, 0.0, 1.0, 42, 9, mode)
        sync()
        assert torch.equal(x, ref) and torch.equal(dsig, ref)
