"""Runs one kernel of the library a few times on a fixed synthetic case, for
profilers (ncu -k <kernel> -c <launches>).  Example:
    python -m paper_1004_3105_gb300.profile_case --kernel polar --n 67108864
Kernels: uniform, b1, polar, batched, reparam_fwd, reparam_bwd.
"""
from __future__ import annotations

import argparse

import numpy as np
import torch

import paper_1004_3105_gb300 as nr
from paper_1004_3105_gb300 import workloads as W

DT = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kernel", required=True,
                    choices=["uniform", "b1", "polar", "batched", "reparam_fwd", "reparam_bwd"])
    ap.add_argument("--n", type=int, default=1 << 26)
    ap.add_argument("--mode", default="accurate", choices=["accurate", "fast"])
    ap.add_argument("--dtype", default="f32", choices=list(DT))
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--streams", type=int, default=1024, help="batched: number of streams")
    ap.add_argument("--methods", default="mixed", choices=["mixed", "b1", "polar"],
                    help="batched: the streams' methods")
    a = ap.parse_args()
    nr.load()
    dev = torch.device("cuda", 0)
    dt = DT[a.dtype]
    if a.kernel in ("uniform", "b1", "polar"):
        out = torch.empty(a.n, dtype=torch.float32 if a.kernel == "uniform" else dt, device=dev)
        ws = nr.polar_workspace(a.n, dev)

        def run():
            if a.kernel == "uniform":
                nr.nrng_uniform(out, W.KEY_MAIN, 0)
            elif a.kernel == "b1":
                nr.nrng_boxmuller(out, 0.0, 1.0, W.KEY_MAIN, 0, a.mode)
            else:
                nr.nrng_polar(out, 0.0, 1.0, W.KEY_MAIN, 0, ws, a.mode)
    elif a.kernel == "batched":
        wl = W.batched_workload(k=a.streams, methods=a.methods, align=4)
        desc = nr.stream_descriptors(wl.offset, wl.n, wl.mu, wl.sigma, wl.key, wl.counter, wl.method)
        d_desc = nr.descriptors_to_device(desc, dev)
        out = torch.empty(wl.total, dtype=dt, device=dev)
        ws = torch.empty(nr.nrng_batched_workspace_size(desc), dtype=torch.uint8, device=dev)

        def run():
            nr.nrng_batched(out, d_desc, len(desc), ws, a.mode)
    else:
        shape = (a.n // 8192, 8192)
        rw = W.reparam_workload(shape=shape)
        mu, sg = torch.from_numpy(rw.mu).to(dev), torch.from_numpy(rw.sigma).to(dev)
        x = torch.empty(shape, device=dev)
        g = torch.from_numpy(rw.w).to(dev)
        dmu, dsg = torch.empty_like(mu), torch.empty_like(sg)

        def run():
            if a.kernel == "reparam_fwd":
                nr.nrng_reparam_fwd(x, mu, sg, W.KEY_REPARAM, 0, a.mode)
            else:
                nr.nrng_reparam_bwd(dmu, dsg, g, W.KEY_REPARAM, 0, a.mode)
    for _ in range(a.reps):
        run()
    torch.cuda.synchronize()
    if a.kernel in ("polar", "batched"):
        st = nr.nrng_get_status(ws)
        if st != 0:
            raise SystemExit(f"device status {st}")
    print(f"ok {a.kernel} n={a.n} mode={a.mode} dtype={a.dtype} reps={a.reps}")


if __name__ == "__main__":
    main()
