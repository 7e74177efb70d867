#!/usr/bin/env python3
"""Benchmark of the normal-variate hot path on GB300, one JSON line on stdout.

A step is one pass over every row of the path on synthetic inputs:
  B1    Box-Muller, N = 2^28 fp32, mu 0, sigma 1, key 0x5EED0001 (accurate)
  P     Polar with order-preserving compaction, same parameters (accurate)
  batch 4096 streams, lengths log-uniform in [1e2, 1e6] (seed 7), mixed B1/P,
        mu ~ U(-2, 2), sigma ~ U(0.1, 3), one persistent launch in a CUDA graph
  rep   reparameterised sample [1024, 8192]: forward x = mu + sigma z, upstream
        gradient of sum(w x^2), backward (z regenerated from its counter)
`value` is normals written per second over the whole step (all ranks).
Every output is larger than L2 (129 MB), so no L2 flush is needed between
steps.  `e2e` repeats the step through the same C-ABI calls with host
buffers: the inputs are copied in from pinned host memory and every output is
copied back, inside the timed region.

--impl reference times the FP64 CPU oracle instead (a deliberately slow
reference, on bounded samples of the same workload).

Multi-GPU (torchrun): every rank runs an independent replica of the step on
its own GPU with its own Philox counter range (the path needs no exchange);
timing is the max over ranks between barriers.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

KEY = 0x5EED0001
N_FULL = 1 << 28
PEAK_FALLBACK_GBS = 6800.0


# ---------------------------------------------------------------- helpers --
def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_counter_base(rank: int, blocks_per_rank: int) -> int:
    """First Philox block of a rank's replica: disjoint ranges per rank."""
    return rank * blocks_per_rank


def max_over_ranks(value: float, world: int) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return PEAK_FALLBACK_GBS, "fallback"


# The sources each recorded kernel is compiled from (its translation unit and
# the headers it includes).
KERNEL_SOURCES = {
    "k_b1": ["k_b1.cu", "nrng_device.cuh", "nrng_internal.h", "h_poly.inc", "sincos_table.inc"],
    "k_polar": ["k_polar.cu", "tiles.cuh", "nrng_device.cuh", "nrng_internal.h", "h_poly.inc", "sincos_table.inc"],
    "k_batched": ["k_batched.cu", "tiles.cuh", "nrng_device.cuh", "nrng_internal.h", "h_poly.inc",
                  "sincos_table.inc"],
}


def _code_only(text: str) -> str:
    """C/C++ source without comments and whitespace: what the compiler sees."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return "".join(text.split())


def source_digest(kernel: str = None) -> str:
    """Digest of a kernel's sources (of all kernel sources when kernel is
    None), comments and whitespace left out, to tell whether recorded
    counters are stale."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1004_3105_gb300", "csrc")
    names = KERNEL_SOURCES.get(kernel) if kernel else None
    for name in sorted(names or os.listdir(csrc)):
        with open(os.path.join(csrc, name), encoding="utf-8", errors="replace") as f:
            h.update(name.encode())
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str):
    """DRAM bytes per launch recorded from an ncu capture of the current
    sources (profiles/ncu_traffic.json), else None."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        rec = d.get(kernel)
        if rec and rec.get("source_digest") == source_digest(kernel):
            return float(rec["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


# --------------------------------------------------------------- clocks ----
class ClockSampler:
    """Samples SM clock, max clock and clock-event reasons through NVML (read
    only) in a thread while the timed region runs."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown", 0x2: "applications_clocks_setting",
               0x1: "gpu_idle"}

    def __init__(self, cuda_index: int, period_s: float = 0.005):
        self.samples, self.reasons, self.max_mhz = [], set(), None
        self.period = period_s
        self.ok = False
        self._stop = threading.Event()
        try:
            self.nvml = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nvml.nvmlInit_v2() != 0:
                return
            self.h = ctypes.c_void_p()
            if not self._handle(cuda_index):
                return
            mx = ctypes.c_uint(0)
            if self.nvml.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0:
                self.max_mhz = int(mx.value)
            self.ok = True
        except OSError:
            pass

    def _handle(self, cuda_index: int) -> bool:
        try:
            import torch
            uuid = "GPU-" + str(torch.cuda.get_device_properties(cuda_index).uuid)
            if self.nvml.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.h)) == 0:
                return True
        except Exception:
            pass
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        idx = cuda_index
        parts = [v.strip() for v in vis.split(",") if v.strip()]
        if parts and cuda_index < len(parts) and parts[cuda_index].isdigit():
            idx = int(parts[cuda_index])
        return self.nvml.nvmlDeviceGetHandleByIndex_v2(idx, ctypes.byref(self.h)) == 0

    def _run(self):
        clk = ctypes.c_uint(0)
        rs = ctypes.c_ulonglong(0)
        while not self._stop.is_set():
            if self.nvml.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(clk)) == 0:
                self.samples.append(int(clk.value))
            if self.nvml.nvmlDeviceGetCurrentClocksEventReasons(self.h, ctypes.byref(rs)) == 0:
                for bit, name in self.REASONS.items():
                    if rs.value & bit and name != "gpu_idle":
                        self.reasons.add(name)
            time.sleep(self.period)

    def __enter__(self):
        if self.ok:
            self._t = threading.Thread(target=self._run, daemon=True)
            self._t.start()
        return self

    def __exit__(self, *exc):
        if self.ok:
            self._stop.set()
            self._t.join()

    def summary(self):
        if not self.ok or not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": sorted(self.reasons),
                    "samples": len(self.samples), "source": "nvml unavailable" if not self.ok else "nvml"}
        return {"sm_mhz": float(np.median(self.samples)), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(self.reasons), "samples": len(self.samples), "source": "nvml"}


def sm_count_of(dev) -> int:
    import torch
    return torch.cuda.get_device_properties(dev).multi_processor_count


def bind_to_gpu_cpus(cuda_index: int):
    """Restricts this process to the host CPUs NVML reports as closest to the
    GPU (read only: a process setting, nothing on the GPU changes), so that
    the pinned host buffers of the end-to-end step are first touched in the
    GPU's local memory.  Returns the CPU list applied, or None."""
    try:
        import torch
        nvml = ctypes.CDLL("libnvidia-ml.so.1")
        if nvml.nvmlInit_v2() != 0:
            return None
        h = ctypes.c_void_p()
        uuid = "GPU-" + str(torch.cuda.get_device_properties(cuda_index).uuid)
        if nvml.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(h)) != 0:
            return None
        words = 64
        mask = (ctypes.c_ulong * words)()
        if nvml.nvmlDeviceGetCpuAffinity(h, words, mask) != 0:
            return None
        cpus = {64 * i + b for i in range(words) for b in range(64) if (mask[i] >> b) & 1}
        cpus &= os.sched_getaffinity(0)
        if not cpus:
            return None
        os.sched_setaffinity(0, cpus)
        return sorted(cpus)
    except (OSError, AttributeError, RuntimeError):
        return None


# ------------------------------------------------------------ GPU workload --
class Step:
    """Buffers and launches of one step of the hot path on one GPU."""

    def __init__(self, rank: int, host_io: bool = False):
        import torch

        import paper_1004_3105_gb300 as nr
        from paper_1004_3105_gb300 import workloads as W
        self.torch, self.nr, self.W = torch, nr, W
        dev = torch.device("cuda", torch.cuda.current_device())
        self.stream = torch.cuda.current_stream()
        # disjoint counter ranges per rank (replicas of the same workload)
        self.base = rank_counter_base(rank, 1 << 40)
        self.out_b1 = torch.empty(N_FULL, dtype=torch.float32, device=dev)
        self.out_p = torch.empty(N_FULL, dtype=torch.float32, device=dev)
        self.ws_p = nr.polar_workspace(N_FULL, dev)
        wl = W.batched_workload(methods="mixed", align=4)
        desc = nr.stream_descriptors(wl.offset, wl.n, wl.mu, wl.sigma, wl.key, wl.counter + np.uint64(self.base),
                                     wl.method)
        self.batch_total, self.batch_k = wl.total, len(desc)
        self.desc_host = desc
        self.desc_dev = nr.descriptors_to_device(desc, dev)
        self.out_batch = torch.empty(wl.total, dtype=torch.float32, device=dev)
        self.ws_batch = torch.empty(nr.nrng_batched_workspace_size(desc), dtype=torch.uint8, device=dev)
        rw = W.reparam_workload()
        self.rep_shape = W.REPARAM_SHAPE
        self.mu = torch.from_numpy(rw.mu).to(dev)
        self.sigma = torch.from_numpy(rw.sigma).to(dev)
        # the loss sum(w x^2) has gradient 2 w x: keep 2w so that it is one multiply
        self.w2 = torch.from_numpy(2.0 * rw.w).to(dev)
        self.x = torch.empty(self.rep_shape, dtype=torch.float32, device=dev)
        self.g = torch.empty_like(self.x)
        self.dmu = torch.empty_like(self.mu)
        self.dsigma = torch.empty_like(self.sigma)
        self.n_rep = int(np.prod(self.rep_shape))
        # autotune the batched launch, then capture it in a graph
        self.batch_cfg, _ = nr.nrng_batched_autotune(self.out_batch, self.desc_dev, self.batch_k, self.ws_batch,
                                                     "accurate", reps=3)
        self.graph = nr.BatchedGraph(self.out_batch, self.desc_dev, self.batch_k, self.ws_batch, "accurate")
        self.host_io = host_io
        if host_io:
            pin = dict(dtype=torch.float32, pin_memory=True)
            self.h_b1 = torch.empty(N_FULL, **pin)
            self.h_p = torch.empty(N_FULL, **pin)
            self.h_batch = torch.empty(wl.total, **pin)
            self.h_x = torch.empty(self.rep_shape, **pin)
            self.h_dmu = torch.empty(self.rep_shape, **pin)
            self.h_dsigma = torch.empty(self.rep_shape, **pin)
            self.h_mu = torch.from_numpy(rw.mu).pin_memory()
            self.h_sigma = torch.from_numpy(rw.sigma).pin_memory()
            self.h_w2 = torch.from_numpy(2.0 * rw.w).pin_memory()
            self.h_desc = torch.from_numpy(desc.view(np.uint8).copy()).pin_memory()
        self.normals_per_step = 2 * N_FULL + self.batch_total + self.n_rep
        # algorithmic Philox blocks of the batched launch: n/4 per B1 stream,
        # n/pi per Polar stream
        self.batch_philox_blocks = float(sum(int(n) / 4 if m == 0 else int(n) / math.pi
                                             for n, m in zip(wl.n, wl.method)))
        # our kernels per step: B1 1, Polar 1, batched 3 (count, fill, main), reparam fwd + bwd 2
        self.our_launches_per_step = 7

    def part_b1(self):
        self.nr.nrng_boxmuller(self.out_b1, 0.0, 1.0, KEY, self.base, "accurate")

    def part_polar(self):
        self.nr.nrng_polar(self.out_p, 0.0, 1.0, KEY, self.base, self.ws_p, "accurate")

    def part_batch(self):
        self.graph.launch()

    def part_reparam(self):
        nr = self.nr
        nr.nrng_reparam_fwd(self.x, self.mu, self.sigma, KEY + 1, self.base, "accurate")
        self.torch.mul(self.w2, self.x, out=self.g)   # dL/dx = 2 w x
        nr.nrng_reparam_bwd(self.dmu, self.dsigma, self.g, KEY + 1, self.base, "accurate")

    PARTS = ("b1", "polar", "batch", "reparam")

    def run_parts(self, events=None):
        for i, name in enumerate(self.PARTS):
            if events is not None:
                events[i][0].record()
            getattr(self, "part_" + name)()
            if events is not None:
                events[i][1].record()

    E2E_COPY_STREAMS = 4

    def _copy_out(self, host, dev, ready):
        """Device -> pinned host copy of `dev`, split into one chunk per copy
        stream, each stream waiting for `ready` (the producing part)."""
        torch = self.torch
        h, d = host.view(-1), dev.view(-1)
        n = d.numel()
        step = (n + len(self.copy_streams) - 1) // len(self.copy_streams)
        for i, cs in enumerate(self.copy_streams):
            lo, hi = i * step, min(n, (i + 1) * step)
            if lo >= hi:
                continue
            cs.wait_event(ready)
            with torch.cuda.stream(cs):
                h[lo:hi].copy_(d[lo:hi], non_blocking=True)

    def run_e2e(self):
        """The step through host buffers: inputs in from pinned memory, every
        output back to pinned memory.  Each part's output is copied out on
        separate copy streams while the next part computes; a part waits for
        the previous step's copies of its own output before overwriting it,
        and the step ends when every copy is done."""
        torch = self.torch
        if not hasattr(self, "copy_streams"):
            self.copy_streams = [torch.cuda.Stream() for _ in range(self.E2E_COPY_STREAMS)]
            self.copied = {}
        main = torch.cuda.current_stream()

        def produce(name, outs, fn):
            for e in self.copied.get(name, ()):
                main.wait_event(e)   # the previous step's copies of these outputs
            fn()
            ready = torch.cuda.Event()
            ready.record(main)
            for host, dev in outs:
                self._copy_out(host, dev, ready)
            ev = []
            for cs in self.copy_streams:
                e = torch.cuda.Event()
                e.record(cs)
                ev.append(e)
            self.copied[name] = ev

        self.mu.copy_(self.h_mu.view(self.rep_shape), non_blocking=True)
        self.sigma.copy_(self.h_sigma.view(self.rep_shape), non_blocking=True)
        self.w2.copy_(self.h_w2.view(self.rep_shape), non_blocking=True)
        self.desc_dev.copy_(self.h_desc, non_blocking=True)
        produce("b1", [(self.h_b1, self.out_b1)], self.part_b1)
        produce("polar", [(self.h_p, self.out_p)], self.part_polar)
        produce("batch", [(self.h_batch, self.out_batch)], self.part_batch)
        produce("reparam", [(self.h_x, self.x), (self.h_dmu, self.dmu), (self.h_dsigma, self.dsigma)],
                self.part_reparam)
        for cs in self.copy_streams:   # the step ends when its copies are done
            e = torch.cuda.Event()
            e.record(cs)
            main.wait_event(e)

    def e2e_bytes(self):
        h2d = 3 * self.n_rep * 4 + self.h_desc.numel()
        d2h = 4 * (2 * N_FULL + self.batch_total + 3 * self.n_rep)
        return h2d, d2h

    def check_status(self):
        nr = self.nr
        for ws in (self.ws_p, self.ws_batch):
            st = nr.nrng_get_status(ws)
            if st != 0:
                raise RuntimeError(f"device status {nr._lib.STATUS.get(st, st)}")


def check_ws(nr, ws):
    """Raises if the workspace's device status word reports an error.  Each
    call clears its workspace first, so the warm-up calls are checked one by
    one: an error in a timed loop would be hidden by the next call."""
    st = nr.nrng_get_status(ws)
    if st != 0:
        raise RuntimeError(f"device status {nr._lib.STATUS.get(st, st)}")


def timed_launches(run, K):
    """Mean ms per launch over K back-to-back launches (events around the
    whole run), plus the median and minimum of the per-launch times (an event
    between consecutive launches)."""
    import torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    ev[0].record()
    for i in range(K):
        run()
        ev[i + 1].record()
    torch.cuda.synchronize()
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(K)]
    return ev[0].elapsed_time(ev[K]) / K, {"ms_median": round(float(np.median(per)), 4),
                                            "ms_min": round(float(np.min(per)), 4)}


def precision_sweep(step, K, W, peak):
    """{B1, Polar} x {accurate, fast} x {f32, bf16, f16} at N = 2^28, then
    Methods B2, B3, P2, R and the two-pass Polar in f32."""
    import torch
    nr = step.nr
    out = {}
    bufs = {torch.float32: step.out_b1, torch.bfloat16: step.out_b1.view(torch.bfloat16)[:N_FULL],
            torch.float16: step.out_b1.view(torch.float16)[:N_FULL]}
    names = {torch.float32: "f32", torch.bfloat16: "bf16", torch.float16: "f16"}
    for method in ("b1", "polar"):
        for mode in ("accurate", "fast"):
            for dt, buf in bufs.items():
                def run():
                    if method == "b1":
                        nr.nrng_boxmuller(buf, 1.5, 0.25, KEY, step.base, mode)
                    else:
                        nr.nrng_polar(buf, 1.5, 0.25, KEY, step.base, step.ws_p, mode)
                for _ in range(W):
                    run()
                    if method == "polar":
                        check_ws(nr, step.ws_p)
                ms, stats = timed_launches(run, K)
                by = N_FULL * buf.element_size()
                gbs = by / (ms * 1e-3) / 1e9
                out[f"{method}_{mode}_{names[dt]}"] = {"ms": round(ms, 4), "normals_per_s": N_FULL / (ms * 1e-3),
                                                       "GB_per_s": round(gbs, 1), "frac_of_hbm": round(gbs / peak, 4),
                                                       **stats}
    # the paper's further methods and the two-pass Polar, f32, same N
    ws_r = torch.empty(nr.nrng_ratio_workspace_size(N_FULL), dtype=torch.uint8, device=step.out_b1.device)
    ws_2 = torch.empty(nr.nrng_polar_twopass_workspace_size(N_FULL), dtype=torch.uint8, device=step.out_b1.device)
    buf = step.out_b1
    variants = {
        "b2_f32": lambda: nr.nrng_boxmuller(buf, 1.5, 0.25, KEY, step.base, "b2"),
        "b3_f32": lambda: nr.nrng_boxmuller_b3(buf, 1.5, 0.25, KEY, step.base),
        "p2_f32": lambda: nr.nrng_polar_p2(buf, 1.5, 0.25, KEY, step.base, step.ws_p),
        "ratio_accurate_f32": lambda: nr.nrng_ratio(buf, 1.5, 0.25, KEY, step.base, ws_r, "accurate"),
        "ratio_fast_f32": lambda: nr.nrng_ratio(buf, 1.5, 0.25, KEY, step.base, ws_r, "fast"),
        "polar_twopass_accurate_f32": lambda: nr.nrng_polar_twopass(buf, 1.5, 0.25, KEY, step.base, ws_2, "accurate"),
        "polar_twopass_fast_f32": lambda: nr.nrng_polar_twopass(buf, 1.5, 0.25, KEY, step.base, ws_2, "fast"),
    }
    checked_ws = {"p2_f32": step.ws_p, "ratio_accurate_f32": ws_r, "ratio_fast_f32": ws_r,
                  "polar_twopass_accurate_f32": ws_2, "polar_twopass_fast_f32": ws_2}
    for name, run in variants.items():
        for _ in range(W):
            run()
            if name in checked_ws:
                check_ws(nr, checked_ws[name])
        ms, stats = timed_launches(run, K)
        gbs = N_FULL * 4 / (ms * 1e-3) / 1e9
        out[name] = {"ms": round(ms, 4), "normals_per_s": N_FULL / (ms * 1e-3), "GB_per_s": round(gbs, 1),
                     "frac_of_hbm": round(gbs / peak, 4), **stats}
    for ws in (ws_r, ws_2):
        st = nr.nrng_get_status(ws)
        if st != 0:
            raise RuntimeError(f"device status {nr._lib.STATUS.get(st, st)}")
    step.check_status()
    return out


def write_ceiling(buf, K, W):
    """What a plain write of the same 1 GiB achieves on this GPU: the
    runtime's cudaMemsetAsync and torch's vectorised fill kernel (a plain
    16-byte store loop), each the mean of K launches after W warm-ups."""
    import torch
    res = {"bytes": buf.numel() * buf.element_size()}
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(W):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(K):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / K
        return round(res["bytes"] / (ms * 1e-3) / 1e9, 1)

    res["fill_GB_per_s"] = timed(lambda: buf.fill_(1.0))
    try:
        rt = ctypes.CDLL("libcudart.so.13")
        rt.cudaMemsetAsync.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p]
        ptr, nbytes, hs = ctypes.c_void_p(buf.data_ptr()), ctypes.c_size_t(res["bytes"]), \
            ctypes.c_void_p(stream.cuda_stream)

        def memset():
            if rt.cudaMemsetAsync(ptr, 0, nbytes, hs) != 0:
                raise RuntimeError("cudaMemsetAsync failed")
        res["memset_GB_per_s"] = timed(memset)
    except (OSError, AttributeError, RuntimeError) as e:
        res["memset_GB_per_s"] = None
        res["memset_note"] = str(e)[:80]
    return res


def philox_ceiling(step, K, W):
    """The rate this GPU draws Philox4x32-10 blocks with no output traffic
    (nrng_philox_ceiling over the 2^26 blocks of a 2^28-normal B1 stream):
    the instruction ceiling every generator here shares."""
    import torch
    nr = step.nr
    acc = torch.zeros(1, dtype=torch.int32, device=step.out_b1.device)
    nblocks = N_FULL // 4

    def run():
        nr.nrng_philox_ceiling(acc, nblocks, KEY, step.base)
    for _ in range(W):
        run()
    ms, stats = timed_launches(run, K)
    return {"nblocks": nblocks, "ms": round(ms, 4), "blocks_per_s": nblocks / (ms * 1e-3), **stats,
            "b1_normals_per_s": 4.0 * nblocks / (ms * 1e-3),
            "polar_normals_per_s": math.pi * nblocks / (ms * 1e-3),
            "source": "measured: nrng_philox_ceiling, CUDA events"}


def tighter_bound(normals_per_s, bytes_per_normal, normals_per_block, ceiling, ph):
    """normals/s against the tighter of the measured write ceiling and the
    measured Philox ceiling (normals_per_block normals per Philox block)."""
    if not ceiling or not ph:
        return None
    wc = max(v for v in (ceiling.get("fill_GB_per_s"), ceiling.get("memset_GB_per_s")) if v)
    b_write = wc * 1e9 / bytes_per_normal
    b_philox = ph["blocks_per_s"] * normals_per_block
    bound, which = (b_write, "hbm write ceiling") if b_write <= b_philox else (b_philox, "philox ceiling")
    return {"bound": which, "normals_per_s": bound, "frac": round(normals_per_s / bound, 4),
            "write_ceiling_normals_per_s": b_write, "philox_ceiling_normals_per_s": b_philox}


def _oracle_work(task):
    """One worker's share of the oracle sample (module level, so that a spawn
    pool can run it): B1 and Polar of n normals each at this worker's own
    counter, and optionally a slice of the batched streams and of the
    reparameterised sample.  Returns the normals produced."""
    import oracle
    from paper_1004_3105_gb300 import workloads as W
    n, counter, reps, extras = task
    normals = 0
    for _ in range(reps):
        oracle.boxmuller(n, 0.0, 1.0, KEY, counter)
        oracle.polar(n, 0.0, 1.0, KEY, counter)
        normals += 2 * n
        if extras:
            wl = W.batched_workload(k=64, methods="mixed")
            oracle.batched(wl.total, wl.as_dict())
            rw = W.reparam_workload(shape=(64, 8192))
            m = rw.mu.size
            x = oracle.reparam_fwd(rw.mu, rw.sigma, m, 1, KEY + 1, counter)
            oracle.reparam_bwd((2 * rw.w.ravel() * x).astype(np.float32), m, 1, KEY + 1, counter)
            normals += wl.total + m
    return normals


class OraclePool:
    """The oracle on every host core: a process pool started with spawn (the
    process already holds a CUDA context, and a forked child of it can hang),
    warmed up before any timing, one task per worker at disjoint counters."""

    def __init__(self, workers=None):
        import multiprocessing as mp
        self.workers = workers or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.workers)
        self.pool.map(_oracle_work, [(1 << 12, 0, 1, True)] * self.workers)   # import, build, load

    def run(self, n, reps, extras):
        tasks = [(n, w * (1 << 40), reps, extras) for w in range(self.workers)]
        t0 = time.perf_counter()
        normals = sum(self.pool.map(_oracle_work, tasks))
        return normals, time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_oracle_sample(seconds_budget: float = 12.0):
    """Times the FP64 oracle on a bounded sample of the step's mix (B1 and
    Polar at equal counts plus a slice of the batched streams and of the
    reparameterised sample): on one core, and on every core of the host with
    one worker process per core."""
    import oracle
    oracle.build()
    n = 1 << 21
    t0 = time.perf_counter()
    _oracle_work((n, 0, 1, True))
    dt1 = time.perf_counter() - t0
    reps = max(1, min(8, int(seconds_budget / 2 / max(dt1, 1e-3))))
    t0 = time.perf_counter()
    normals1 = _oracle_work((n, 0, reps, True))
    dt1 = time.perf_counter() - t0
    one = {"value": normals1 / dt1, "unit": "normals/s", "cores": 1, "seconds": round(dt1, 2)}
    sample = (f"{reps} x (B1 2^21 + Polar 2^21 + 64 batched streams + reparam fwd+bwd [64, 8192]) per worker, "
              f"FP64 C oracle, disjoint counters per worker")
    try:
        pool = OraclePool()
        normals, dt = pool.run(n, reps, True)
        pool.close()
        return {"value": normals / dt, "unit": "normals/s", "cores": pool.workers, "kind": "oracle",
                "sample": sample, "seconds": round(dt, 2), "single_core": one}
    except Exception as e:   # no pool on this host: the single-core figure stands
        log(f"oracle pool unavailable ({e}); single-core baseline only")
        return {"value": one["value"], "unit": "normals/s", "cores": 1, "kind": "oracle", "sample": sample,
                "seconds": one["seconds"]}


def timed_flushed(run, K, flush):
    """Median and minimum ms of K launches, each after an L2 flush (outside
    the events): for outputs that fit in L2."""
    import torch
    per = []
    for _ in range(K):
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        per.append(e0.elapsed_time(e1))
    return float(np.median(per)), {"ms_median": round(float(np.median(per)), 4), "ms_min": round(float(np.min(per)), 4)}


def configs_sweep(step, K, warm, peak):
    """The smaller single-stream cases (B1 at 2^20, which fits in L2 and is
    timed per launch after an L2 flush; B1 and Polar at 2^26), and the
    4096-stream batched workload with every stream B1, every stream Polar, and
    mixed, each as one graph launch in the configuration the step uses,
    against a single stream of the same total length."""
    import torch
    nr = step.nr
    dev = step.out_b1.device
    out = {}
    flush_buf = torch.empty(64 << 20, dtype=torch.float32, device=dev)   # 256 MB > L2
    ws_small = nr.polar_workspace(1 << 26, dev)
    cases = {
        "c1_b1_accurate_2p20": (1 << 20, lambda b: nr.nrng_boxmuller(b, 0.0, 1.0, KEY, step.base, "accurate")),
        "c2_b1_accurate_2p26": (1 << 26, lambda b: nr.nrng_boxmuller(b, 0.0, 1.0, KEY, step.base, "accurate")),
        "c2_polar_accurate_2p26": (1 << 26, lambda b: nr.nrng_polar(b, 0.0, 1.0, KEY, step.base, ws_small,
                                                                    "accurate")),
    }
    for name, (n, call) in cases.items():
        buf = step.out_b1[:n]
        for _ in range(warm):
            call(buf)
        check_ws(nr, ws_small)
        if n * 4 < (129 << 20):
            ms, stats = timed_flushed(lambda: call(buf), K, flush_buf.zero_)
        else:
            ms, stats = timed_launches(lambda: call(buf), K)
        check_ws(nr, ws_small)
        gbs = n * 4 / (ms * 1e-3) / 1e9
        out[name] = {"n": n, "ms": round(ms, 4), "normals_per_s": n / (ms * 1e-3), "GB_per_s": round(gbs, 1),
                     "frac_of_hbm": round(gbs / peak, 4), **stats}
    del flush_buf
    for methods in ("b1", "polar", "mixed"):
        wl = step.W.batched_workload(methods=methods, align=4)
        desc = nr.stream_descriptors(wl.offset, wl.n, wl.mu, wl.sigma, wl.key, wl.counter + np.uint64(step.base),
                                     wl.method)
        normals = int(wl.n.sum())
        buf = torch.empty(wl.total, dtype=torch.float32, device=dev)
        ws = torch.empty(nr.nrng_batched_workspace_size(desc), dtype=torch.uint8, device=dev)
        dd = nr.descriptors_to_device(desc, dev)
        g = nr.BatchedGraph(buf, dd, len(desc), ws, "accurate")
        for _ in range(warm):
            g.launch()
        check_ws(nr, ws)
        ms, stats = timed_launches(g.launch, K)
        check_ws(nr, ws)
        g.close()
        gbs = normals * 4 / (ms * 1e-3) / 1e9
        entry = {"streams": len(desc), "normals": normals, "ms": round(ms, 4), "normals_per_s": normals / (ms * 1e-3),
                 "GB_per_s": round(gbs, 1), "frac_of_hbm": round(gbs / peak, 4), **stats}
        if methods != "mixed":
            one = buf[:normals]
            ws_one = nr.polar_workspace(normals, dev) if methods == "polar" else None
            if methods == "b1":
                def single():
                    nr.nrng_boxmuller(one, 0.0, 1.0, KEY, step.base, "accurate")
            else:
                def single():
                    nr.nrng_polar(one, 0.0, 1.0, KEY, step.base, ws_one, "accurate")
            for _ in range(warm):
                single()
            ms1, _ = timed_launches(single, K)
            if ws_one is not None:
                check_ws(nr, ws_one)
            entry["single_stream_ms"] = round(ms1, 4)
            entry["single_stream_over_batched"] = round(ms1 / ms, 4)
        out[f"batched_{methods}"] = entry
        del buf, ws, dd
    step.check_status()
    return out


# ------------------------------------------------------------------- arms --
def workload_config(world, batch_total, rep_shape):
    """The `config` object of both arms' JSON lines: the step's workload."""
    return {"workload": "B1 2^28 fp32 + Polar 2^28 fp32 (accurate, mu 0, sigma 1, key 0x5EED0001) + "
                        "4096 batched streams (seed 7, mixed, graph) + reparam fwd+bwd [1024, 8192]",
            "N": N_FULL, "batched_normals": int(batch_total), "reparam_shape": list(rep_shape),
            "l2": "outputs > L2 (1 GiB per single-stream kernel, 1.8 GB batched); the reparam part's 32 MiB "
                  "arrays are evicted by the 3.7 GB the other parts write each step; no flush",
            "parallelism": f"replicas x{world}"}


def bench_reference(args):
    """The FP64 oracle, as it stands, on every host core: each step is a
    bounded sample of the step's mix (B1 and Polar at 2^20 each, a 64-stream
    slice of the batched workload and a [64, 8192] slice of the reparameterised
    sample, per worker, at disjoint counters)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1004_3105_gb300 import workloads as W
    oracle.build()
    n = 1 << 20
    pool = OraclePool()
    for _ in range(args.warmup):
        pool.run(n, 1, True)
    total, dt = 0, 0.0
    for _ in range(args.steps):
        normals, t = pool.run(n, 1, True)
        total += normals
        dt += t
    pool.close()
    value = total / dt
    per_step = total // max(1, args.steps)
    sample = (f"per step and worker: B1 2^20 + Polar 2^20 + 64 batched streams + reparam fwd+bwd [64, 8192] "
              f"(FP64 C oracle, {pool.workers} workers, disjoint counters); {per_step} normals per step")
    wl = W.batched_workload(methods="mixed", align=4)
    line = {
        "impl": "reference", "metric": "normals/s", "value": value, "unit": "normals/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.gpus, wl.total, W.REPARAM_SHAPE),
        "cpu_baseline": {"value": value, "unit": "normals/s", "cores": pool.workers, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "normals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def bench_ours(args):
    rank, world, local = dist_env()
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    import paper_1004_3105_gb300 as nr
    nr.load()
    cpus_all = os.sched_getaffinity(0)
    cpus_gpu = bind_to_gpu_cpus(local) if not args.no_e2e else None
    step = Step(rank, host_io=not args.no_e2e)
    torch.cuda.synchronize()

    # ---- device-resident timed region
    for _ in range(args.warmup):
        step.run_parts()
        step.check_status()   # per warm-up step: the next step's clear would hide an error
    torch.cuda.synchronize()
    K = args.steps
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in Step.PARTS] for _ in range(K)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        start.record()
        for k in range(K):
            step.run_parts(ev[k])
        stop.record()
        torch.cuda.synchronize()
    barrier(world)
    step.check_status()
    ms_local = start.elapsed_time(stop)
    ms = max_over_ranks(ms_local, world)
    part_ms = {name: float(np.mean([ev[k][i][0].elapsed_time(ev[k][i][1]) for k in range(K)]))
               for i, name in enumerate(Step.PARTS)}
    value = world * K * step.normals_per_step / (ms * 1e-3)

    # ---- end to end through host buffers
    e2e = None
    if not args.no_e2e:
        Ke = max(2, min(K, args.e2e_steps))
        for _ in range(2):
            step.run_e2e()
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(Ke):
            step.run_e2e()
        e1.record()
        torch.cuda.synchronize()
        barrier(world)
        ems = max_over_ranks(e0.elapsed_time(e1), world)
        h2d, d2h = step.e2e_bytes()
        e2e = {"value": world * Ke * step.normals_per_step / (ems * 1e-3), "unit": "normals/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": Ke,
               "ms_per_step": ems / Ke, "d2h_GB_per_s": round(d2h / (ems / Ke * 1e-3) / 1e9, 1),
               "host_cpus": (f"{len(cpus_gpu)} GPU-local cpus" if cpus_gpu else "unbound")}

    # ---- roofline of the dominant kernel and per-part rates
    peak, peak_src = measured_peaks()
    alg_bytes = {"b1": 4 * N_FULL, "polar": 4 * N_FULL, "batch": 4 * step.batch_total,
                 "reparam": 24 * step.n_rep}   # fwd 12 B/elem; bwd reads g, writes dmu, dsigma: 12 B/elem
    kernel_names = {"b1": "k_b1", "polar": "k_polar", "batch": "k_batched", "reparam": "k_reparam"}
    parts = {}
    for name in Step.PARTS:
        t = part_ms[name] * 1e-3
        gbs = alg_bytes[name] / t / 1e9
        parts[name] = {"ms": round(part_ms[name], 4), "GB_per_s": round(gbs, 1),
                       "frac_of_hbm": round(gbs / peak, 4)}
    parts["b1"]["normals_per_s"] = N_FULL / (part_ms["b1"] * 1e-3)
    parts["polar"]["normals_per_s"] = N_FULL / (part_ms["polar"] * 1e-3)
    parts["batch"]["normals_per_s"] = step.batch_total / (part_ms["batch"] * 1e-3)
    parts["batch"]["config"] = list(nr.nrng_batched_config_info(step.batch_cfg))
    parts["reparam"]["fwd_bwd_per_s"] = 1.0 / (part_ms["reparam"] * 1e-3)
    dom = max(("b1", "polar", "batch"), key=lambda nm: part_ms[nm])
    t_dom = part_ms[dom] * 1e-3
    achieved = alg_bytes[dom] / t_dom / 1e9
    roofline = {"kernel": kernel_names[dom], "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": peak_src,
                "traffic": recorded_traffic(kernel_names[dom]),
                "algorithmic_bytes_per_launch": alg_bytes[dom]}
    # ---- precision sweep at N = 2^28 (mu 1.5, sigma 0.25): each variant timed
    # alone with CUDA events (mean of K launches after W warm-ups), not part of
    # the step
    sweep = {}
    ceiling = None
    ph = None
    if not args.no_sweep:
        sweep = precision_sweep(step, K, args.warmup, peak)
        sweep.update(configs_sweep(step, K, args.warmup, peak))
        ceiling = write_ceiling(step.out_b1, K, args.warmup)
        ph = philox_ceiling(step, K, args.warmup)
        # every sweep row against the tighter of the two measured ceilings
        per_block = {"b1": 4.0, "b2": 4.0, "b3": 8.0 / 3.0, "polar": math.pi, "p2": math.pi,
                     "ratio": 2.0 * (math.pi * math.e) ** 0.5 / 4.0}
        for name, row in sweep.items():
            if "normals_per_s" not in row or name.startswith("batched") or name.startswith("c1_"):
                continue
            head = name.split("_")[0] if not name.startswith("c2_") else name.split("_")[1]
            nb = 2 if ("bf16" in name or "f16" in name) else 4
            tb = tighter_bound(row["normals_per_s"], nb, per_block.get(head, 4.0), ceiling, ph)
            if tb:
                row["frac_of_tighter"] = tb["frac"]
                row["tighter_bound"] = tb["bound"]

    def kernel_roofline(part, kernel, per_block):
        t = part_ms[part] * 1e-3
        achieved = alg_bytes[part] / t / 1e9
        d = {"kernel": kernel, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
             "frac": round(achieved / peak, 4), "peak_source": peak_src, "traffic": recorded_traffic(kernel),
             "algorithmic_bytes_per_launch": alg_bytes[part]}
        if ceiling:
            wc = max(v for v in (ceiling.get("fill_GB_per_s"), ceiling.get("memset_GB_per_s")) if v)
            d["write_ceiling_GB_per_s"] = wc
            d["frac_of_write_ceiling"] = round(achieved / wc, 4)
        tb = tighter_bound(N_FULL / t, 4, per_block, ceiling, ph)
        if tb:
            d["tighter"] = tb
        return d
    roofline_b1 = kernel_roofline("b1", "k_b1", 4.0)
    roofline_polar = kernel_roofline("polar", "k_polar", math.pi)

    # The same kernel against the Philox ceiling: the measured rate of
    # nrng_philox_ceiling when the sweep ran, else derived (20 32x32->64
    # products a block at 64 products a clock per SM, two per wide product:
    # 1.6 blocks a clock per SM).  Algorithmic blocks: n/4 per B1 stream, n/pi
    # per Polar stream (n/2 pairs at acceptance pi/4, two candidates a block).
    sm_mhz = clocks.summary().get("sm_mhz") or 2070.0
    alg_blocks = {"b1": N_FULL / 4, "polar": N_FULL / math.pi, "batch": step.batch_philox_blocks}
    if ph:
        floor, floor_src = ph["blocks_per_s"], "measured: nrng_philox_ceiling over 2^26 blocks, CUDA events"
    else:
        floor = sm_count_of(torch.cuda.current_device()) * sm_mhz * 1e6 * 1.6
        floor_src = f"derived: SMs x {sm_mhz:.0f} MHz x 1.6 blocks/clock/SM"
    roofline_philox = {"kernel": kernel_names[dom], "bound": "alu", "unit": "Philox blocks/s",
                       "achieved": alg_blocks[dom] / t_dom, "peak": floor,
                       "frac": round(alg_blocks[dom] / t_dom / floor, 4), "peak_source": floor_src}

    cpu = None
    os.sched_setaffinity(0, cpus_all)   # the CPU baseline uses every core
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": "normals/s", "value": value, "unit": "normals/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (Philox4x32-10 streams; seeded PCG64 inputs)",
            "config": workload_config(world, step.batch_total, step.rep_shape),
            "parts": parts, "sweep": sweep, "write_ceiling": ceiling, "philox_ceiling": ph, "roofline": roofline,
            "roofline_b1": roofline_b1, "roofline_polar": roofline_polar, "roofline_philox": roofline_philox,
            "clocks": clocks.summary(),
            "e2e": e2e, "gpu_launches": K * step.our_launches_per_step, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    args = ap.parse_args()
    if args.warmup < 3:
        log("warmup raised to 3 (timing rule)")
        args.warmup = 3
    if args.impl == "reference":
        return bench_reference(args)
    return bench_ours(args)


if __name__ == "__main__":
    sys.exit(main())
