"""Device-side error paths, made without faulting the GPU: a Polar tile that
never publishes its status (a flag that nothing sets) makes its successors'
bounded look-back waits run out, and a capped tile budget makes a stream run
out of tiles.  Each runs in a child process whose environment turns the test
hook on; the kernel records the status word and returns, and the context
stays usable for the next call."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import os, sys, time
    sys.path.insert(0, {root!r})
    import torch, numpy as np
    import paper_1004_3105_gb300 as nr
    import oracle
    n = 1 << 22
    out = torch.empty(n, device="cuda")
    ws = nr.polar_workspace(n)
    t0 = time.time()
    nr.nrng_polar(out, 0.0, 1.0, 5, 0, ws)
    st = nr.nrng_get_status(ws)
    dt = time.time() - t0
    print("STATUS", st, "SECONDS", round(dt, 3))
    # hook off: the same context still generates the right stream
    os.environ.pop("NRNG_DEBUG_SILENT_TILE", None)
    os.environ.pop("NRNG_DEBUG_POLAR_TILES", None)
    m = 100001
    out2 = torch.empty(m, device="cuda")
    nr.nrng_polar(out2, 0.0, 1.0, 5, 0, ws)
    st2 = nr.nrng_get_status(ws)
    ref = oracle.polar(m, 0.0, 1.0, 5, 0)[0]
    err = float(np.max(np.abs(out2.cpu().numpy() - ref) / np.maximum(1, np.abs(ref))))
    print("AFTER", st2, "ERR", err)
""")


def run_child(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    vals = {}
    for line in r.stdout.splitlines():
        parts = line.split()
        if parts and parts[0] in ("STATUS", "AFTER"):
            vals[parts[0]] = parts
    return vals


def test_lookback_timeout_is_reported():
    v = run_child({"NRNG_DEBUG_SILENT_TILE": "3", "NRNG_LOOKBACK_SPIN_LIMIT_MS": "200"})
    assert int(v["STATUS"][1]) == 6            # NRNG_ERR_TIMEOUT
    assert float(v["STATUS"][3]) < 30.0        # bounded: one wait limit, not a hang
    assert int(v["AFTER"][1]) == 0 and float(v["AFTER"][3]) < 4e-6


def test_tile_budget_exhaustion_is_reported():
    v = run_child({"NRNG_DEBUG_POLAR_TILES": "5"})
    assert int(v["STATUS"][1]) == 7            # NRNG_ERR_EXHAUSTED
    assert int(v["AFTER"][1]) == 0 and float(v["AFTER"][3]) < 4e-6
