"""The host side of the multi-GPU bench path, on CPU with two gloo ranks.

Instances shard across ranks with no data-path exchange: each rank solves its
own independently seeded column, the job's time is the slowest rank's, and the
whole-job rate is the units all ranks processed over that time.  The only
collective is the max over ranks of the timings."""
import json
import os
import socket
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
import paper_2606_04725_gb300.inputs as I
rank, world, _ = bench._dist()
dist.init_process_group("gloo", rank=rank, world_size=world)
wl = I.WORKLOADS[bench.WORKLOAD]
seed = bench.rank_seed(wl, rank)
x0 = I.distillation_x0(wl["N"], wl["Nf"], seed)
# rank r "took" 1 + r seconds for 10 re-solves
secs = 1.0 + rank
out = {"rank": rank, "seed": seed, "x0": x0.tolist(),
       "max": bench.max_over_ranks(secs, world),
       "rate": bench.whole_job_rate(10, secs, world)}
dist.barrier()
dist.destroy_process_group()
print(json.dumps(out))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    env.pop("CUDA_VISIBLE_DEVICES", None)
    return env


def test_two_ranks_shard_and_take_the_slowest_time():
    world, port = 2, _free_port()
    procs = [subprocess.Popen([sys.executable, "-c", RANK_SCRIPT, ROOT], env=_env(r, world, port),
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for r in range(world)]
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=240)
        assert p.returncode == 0, e[-2000:]
        outs.append(json.loads(o.strip().splitlines()[-1]))
    outs.sort(key=lambda d: d["rank"])
    # every rank sees the slowest rank's time and the same whole-job rate
    for d in outs:
        assert d["max"] == 2.0
        assert d["rate"] == world * 10 / 2.0
    # the ranks solve different columns
    assert outs[0]["seed"] != outs[1]["seed"]
    assert not np.allclose(outs[0]["x0"], outs[1]["x0"])


def test_one_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(47, 0.5, 1) == 94.0


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the oracle arm prints from rank 0; the other ranks exit 0
    without work or output."""
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=_env(1, 2, _free_port()), capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""
