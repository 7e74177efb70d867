"""The benchmark's multi-rank logic on CPU (gloo, world_size 2): each rank's
replica draws from a disjoint Philox counter range, and the step time is the
maximum over ranks.  The generators themselves need no exchange."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    base = bench.rank_counter_base(r, 1 << 40)
    t = bench.max_over_ranks(10.0 + r, w)   # rank r "took" 10 + r ms
    bench.barrier(w)
    q.put((r, base, t))
    dist.destroy_process_group()


def test_two_rank_partition_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, b0, t0), (r1, b1, t1) = res
    assert (r0, r1) == (0, 1)
    assert t0 == t1 == 11.0                 # max over ranks
    # disjoint counter ranges, each far larger than one step's Polar budget
    import sys
    sys.path.insert(0, ROOT)
    from paper_1004_3105_gb300 import _lib
    lib = _lib.load(build_if_missing=True)
    import ctypes
    blocks = ctypes.c_uint64(0)
    assert lib.nrng_polar_max_blocks(1 << 28, ctypes.byref(blocks)) == 0
    assert b1 - b0 >= blocks.value + (1 << 26)
