"""The reference arm of bench.py (the FP64 oracle on the host cores), which
needs no GPU: its one JSON line carries every key of the bench contract, the
same config object as the GPU arm, and a cpu_baseline and an e2e object that
describe the same run; under a multi-rank launch only rank 0 prints."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e")


def run_reference(env_extra=None):
    env = dict(os.environ, **(env_extra or {}))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout


def test_reference_arm_json_line():
    out = run_reference()
    line = json.loads(out.strip().splitlines()[-1])
    for k in KEYS:
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == "normals/s" and line["unit"] == "normals/s"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["warmup"] >= 3
    from paper_1004_3105_gb300 import workloads as W
    wl = W.batched_workload(methods="mixed", align=4)
    assert line["config"] == bench.workload_config(1, wl.total, W.REPARAM_SHAPE)
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == line["value"] and cpu["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "normals/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_print_nothing():
    out = run_reference({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert out.strip() == ""


def test_source_digest_ignores_comments_and_tracks_code():
    a = "int f(int x) {\n    return x + 1;   // one more\n}\n/* block\n comment */\n"
    b = "int f(int x){return x+1;}"
    c = "int f(int x) { return x + 2; }"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)

