"""Host side of a run on several GPUs (independent replicas, one process per
GPU): two gloo ranks on the CPU, launched as the launcher would (RANK,
WORLD_SIZE, LOCAL_RANK, MASTER_ADDR=127.0.0.1), agree on the slowest rank's time
and on the whole-job throughput."""
import json
import os
import socket
import subprocess
import sys

from conftest import ROOT

WORKER = r"""
import json, sys
import torch.distributed as dist
from paper_2507_21791_gb300 import replicas
world, rank, local = replicas.dist_env()
dist.init_process_group("gloo")
ms = replicas.max_over_ranks(10.0 + 5.0 * rank)      # rank 1 is the slow one
gbs = replicas.whole_job_gbs(world, 1e9, ms)
dist.barrier()
print(json.dumps({"rank": rank, "world": world, "local": local, "ms": ms, "gbs": gbs}))
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_agree_on_max_time_and_whole_job_value():
    port = free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["world"] == 2 and o["local"] == o["rank"]
        assert o["ms"] == 15.0                       # the max over ranks, on every rank
        assert abs(o["gbs"] - 2 * 1e9 / 15e-3 / 1e9) < 1e-9


def test_single_process_defaults():
    from paper_2507_21791_gb300 import replicas

    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    old = dict(os.environ)
    try:
        os.environ.clear()
        os.environ.update(env)
        assert replicas.dist_env() == (1, 0, 0)
        assert replicas.max_over_ranks(3.5) == 3.5
        assert replicas.whole_job_gbs(1, 2e9, 1000.0) == 2.0
    finally:
        os.environ.clear()
        os.environ.update(old)
