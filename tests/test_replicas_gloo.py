"""Multi-GPU is replicas only (views are independent through the fit step and
this build has no collective on the data path): N ranks each time the same
steps; the job's time is the slowest rank's and its throughput all ranks'
iterations over that time. The rank-side aggregation runs here on two gloo
ranks on the CPU; the reference arm does its work on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["ROOT"])
import torch.distributed as dist
import bench
rank = int(os.environ["RANK"])
dist.init_process_group("gloo")
ms_total = [40.0, 55.0][rank]  # this rank's timed total over 10 steps
ms, value = bench.aggregate(ms_total, 10, 2, "cpu")
print(json.dumps({"rank": rank, "ms": ms, "value": value}))
dist.destroy_process_group()
"""


def _launch(code, world, extra_env=None):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, ROOT=ROOT, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), **(extra_env or {}))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(out)
    return outs


def test_two_gloo_ranks_take_the_slowest_rank():
    outs = [json.loads(o.strip().splitlines()[-1]) for o in _launch(WORKER, 2)]
    for o in outs:
        assert o["ms"] == pytest.approx(5.5)           # the slower rank: 55 ms / 10 steps
        assert o["value"] == pytest.approx(2 * 1000 / 5.5)  # both ranks' iterations over that time


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun, ranks other than 0 exit 0 without work or output."""
    code = ("import os, sys; sys.path.insert(0, os.environ['ROOT']); sys.argv = ['bench.py', '--impl', 'reference', "
            "'--gpus', '2', '--steps', '1', '--warmup', '1']; import bench; bench.main()")
    env = dict(os.environ, ROOT=ROOT, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""
