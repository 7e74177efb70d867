"""Concurrent host threads through the C ABI.  Each thread makes its own
calls (B1, Polar with continuation, R, batched) on its own CUDA stream with
its own buffers and workspaces, all threads starting together; every result
and status equals what the same calls give when made alone, one after the
other.  The ABI's per-process state (cached occupancies and SM counts, the
batched configuration table) is shared by the threads."""
import threading

import numpy as np
import pytest
import torch

import paper_1004_3105_gb300 as nr
from paper_1004_3105_gb300 import workloads as W

pytestmark = pytest.mark.gpu
THREADS = 4
REPS = 6


class Job:
    """One thread's buffers and calls."""

    def __init__(self, i):
        dev = torch.device("cuda", 0)
        self.i = i
        self.key = 0x7A000000 + i
        self.n = 1_000_003 + 4099 * i
        self.b1 = torch.empty(self.n, dtype=torch.float32, device=dev)
        self.p = torch.empty(self.n, dtype=torch.float32, device=dev)
        self.r = torch.empty(self.n // 2 + 1, dtype=torch.float32, device=dev)
        self.ws_p = nr.polar_workspace(self.n, dev)
        self.ws_r = nr.ratio_workspace(self.r.numel(), dev)
        self.next_p = torch.zeros(1, dtype=torch.int64, device=dev)
        wl = W.batched_workload(k=64 + 16 * i, len_lo=10, len_hi=60000, seed=100 + i)
        desc = nr.stream_descriptors(wl.offset, wl.n, wl.mu, wl.sigma, wl.key, wl.counter, wl.method)
        self.k = len(desc)
        self.desc = nr.descriptors_to_device(desc, dev)
        self.bo = torch.empty(wl.total, dtype=torch.float32, device=dev)
        self.ws_b = torch.empty(nr.nrng_batched_workspace_size(desc), dtype=torch.uint8, device=dev)

    def run(self, stream):
        statuses = []
        for rep in range(REPS):
            mode = "accurate" if rep % 2 == 0 else "fast"
            nr.nrng_boxmuller(self.b1, 0.5, 2.0, self.key, rep, mode, stream=stream)
            nr.nrng_polar(self.p, -1.0, 0.5, self.key, 1000 * rep, self.ws_p, mode, next_counter=self.next_p,
                          stream=stream)
            statuses.append(nr.nrng_get_status(self.ws_p, stream))
            nr.nrng_ratio(self.r, 0.0, 1.0, self.key + 1, rep, self.ws_r, mode, stream=stream)
            statuses.append(nr.nrng_get_status(self.ws_r, stream))
            nr.nrng_batched(self.bo, self.desc, self.k, self.ws_b, mode, stream=stream)
            statuses.append(nr.nrng_get_status(self.ws_b, stream))
        stream.synchronize()
        return statuses, [t.cpu().clone() for t in (self.b1, self.p, self.r, self.bo, self.next_p)]


def test_concurrent_threads_match_sequential():
    jobs = [Job(i) for i in range(THREADS)]
    torch.cuda.synchronize()
    # alone, one after the other
    want = [job.run(torch.cuda.Stream()) for job in jobs]
    for job in jobs:
        for t in (job.b1, job.p, job.r, job.bo):
            t.fill_(float("nan"))
    torch.cuda.synchronize()

    got = [None] * THREADS
    errors = []
    start = threading.Barrier(THREADS)

    def worker(i):
        try:
            stream = torch.cuda.Stream()
            start.wait()
            got[i] = jobs[i].run(stream)
        except Exception as e:   # reported below, in the main thread
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(THREADS)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for i in range(THREADS):
        st_want, out_want = want[i]
        st_got, out_got = got[i]
        assert st_got == [0] * len(st_got) and st_want == st_got
        for a, b in zip(out_want, out_got):
            assert torch.equal(a, b), f"thread {i}"
