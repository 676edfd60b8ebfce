"""The N > 1 path of bench.py on CPU: two gloo ranks agree on the slowest
rank's time and on the whole-job throughput; the reference arm prints only on
rank 0."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
dist.init_process_group("gloo")
import bench
r = dist.get_rank()
ms = 100.0 + 50.0 * r                      # rank 1 is the slow one
mx = bench.max_over_ranks(ms)
v = bench.job_throughput(dist.get_world_size(), 1e12, 2, mx)
print(json.dumps({{"rank": r, "max": mx, "value": v}}), flush=True)
dist.destroy_process_group()
"""


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def run_ranks(code, n=2, extra_env=None):
    port = free_port()
    procs = []
    for r in range(n):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(n), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), **(extra_env or {}))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    return [o for o, _ in outs]


def test_two_ranks_agree_on_max_time_and_job_throughput():
    import json
    outs = [json.loads(o.strip().splitlines()[-1]) for o in run_ranks(WORKER.format(root=ROOT))]
    assert all(o["max"] == 150.0 for o in outs)
    # 2 ranks x 1 TFLOP x 2 steps in 150 ms
    assert all(o["value"] == pytest.approx(2 * 1e12 * 2 / 0.150 / 1e12) for o in outs)


def test_reference_arm_prints_on_rank_zero_only():
    code = ("import sys; sys.argv = ['bench.py', '--impl', 'reference', '--gpus', '2', '--steps', '1', "
            "'--warmup', '3', '--ref-budget', '0.05']; sys.path.insert(0, %r); import bench; bench.main()" % ROOT)
    outs = run_ranks(code)
    assert '"impl": "reference"' in outs[0]
    assert outs[1].strip() == ""
