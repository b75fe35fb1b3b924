"""The multi-rank path of bench.py on CPU ranks (gloo, world size 2): timing is the max over
ranks, throughput is summed over replicas, and only rank 0 reports.  Trajectories are
independent ODEs, so ranks are replicas and exchange nothing on the data path."""
import json
import os
import socket
import subprocess
import sys

import pytest


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
rank = int(os.environ["RANK"]); world = int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo")
local_ms = 100.0 + 50.0 * rank
ms = bench.reduce_max(local_ms, world)
bench.barrier(world)
acc_local = 12 * (rank + 1)
value = world * acc_local / (ms / 1e3)
print(json.dumps({{"rank": rank, "ms": ms, "value": value}}), flush=True)
dist.destroy_process_group()
"""


def _launch(code, world):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(out)
    return outs


def test_max_over_ranks_timing_with_gloo():
    outs = _launch(WORKER.format(root=ROOT), 2)
    res = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    assert all(r["ms"] == 150.0 for r in res)                 # max over ranks, seen by every rank


def test_reference_arm_runs_on_rank_zero_only():
    code = ("import sys; sys.path.insert(0, %r); import bench, argparse\n"
            "a = argparse.Namespace(steps=1, gpus=2)\n"
            "sys.exit(bench.run_reference(a, rank=1, world=2))" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line_carries_the_contract_keys(capsys):
    """bench.py --impl reference on one rank: the oracle timed on a bounded sample (here a small
    shape so the test stays short), printed as one JSON line with the keys the contract names."""
    import bench
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "1", "--o", "2", "--v", "6"]) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["warmup"] == 1 and line["steps"] == 1
    # each step is one bounded sample (a T-residual), so steps x ms_per_step is the timed CPU work
    assert line["step_kind"].startswith("sample") and line["ms_per_step"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert "o=2 v=6" in line["config"]["workload"]
