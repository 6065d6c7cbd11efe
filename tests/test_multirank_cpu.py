"""The host side of the multi-GPU bench path, on CPU with two gloo ranks.

The batch's instances shard across ranks with no data-path exchange: each rank
takes a contiguous instance range, the ranges balanced by the factorization
work of each instance (from the host-only structure analysis); the job's time
is the slowest rank's, and the whole-job rate is the units all ranks processed
over that time.  The only collectives are the max and sum of the timings."""
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
import numpy as np
import torch
import torch.distributed as dist
import bench
import paper_2606_04725_gb300 as P
import paper_2606_04725_gb300.inputs as I
from paper_2606_04725_gb300.partition import instance_weights, rank_slice
rank, world, _ = bench._dist()
dist.init_process_group("gloo", rank=rank, world_size=world)
wl = I.WORKLOADS[bench.WORKLOAD]
hz, x0s, sps = bench.batch_inputs(wl)
w = instance_weights(P.MODEL_DISTILLATION, hz, N=wl["N"], Nf=wl["Nf"])
i0, i1 = rank_slice(w, rank, world)
# every rank sees every rank's range
got = [None] * world
dist.all_gather_object(got, [i0, i1])
# a rank "takes" time in proportion to its share of the factorization work
secs = float(w[i0:i1].sum() / w.sum())
out = {"rank": rank, "slices": got, "weights": w.tolist(), "secs": secs,
       "max": bench.max_over_ranks(secs, world),
       "rate": bench.whole_job_rate(10 * (i1 - i0), secs, world)}
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


def test_two_ranks_split_the_batch_and_take_the_slowest_time():
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
    w = np.array(outs[0]["weights"])
    slices = outs[0]["slices"]
    assert all(d["slices"] == slices for d in outs)
    # contiguous ranges that cover every instance exactly once
    assert slices[0][0] == 0 and slices[-1][1] == w.size
    assert all(a[1] == b[0] and a[0] < a[1] for a, b in zip(slices, slices[1:] + [[w.size, w.size + 1]]))
    # balanced by factorization work: no rank above its share by more than one instance
    loads = [w[a:b].sum() for a, b in slices]
    assert max(loads) <= w.sum() / world + w.max()
    # the job's time is the slowest rank's; the rate counts every rank's units
    for d in outs:
        assert d["max"] == max(o["secs"] for o in outs)
        assert abs(d["rate"] - 10 * w.size / d["max"]) <= 1e-9 * d["rate"]


def test_one_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(47, 0.5, 1) == 94.0


def test_contiguous_partition_edge_cases():
    from paper_2606_04725_gb300.partition import contiguous_partition
    import pytest
    assert contiguous_partition([1.0] * 8, 4) == [0, 2, 4, 6, 8]
    assert contiguous_partition([5.0, 1.0, 1.0, 1.0], 2) == [0, 1, 4]
    assert contiguous_partition([1.0, 1.0], 2) == [0, 1, 2]            # one instance per rank
    assert contiguous_partition([0.0, 0.0, 0.0], 3) == [0, 1, 2, 3]     # no weight: still non-empty ranges
    assert contiguous_partition([100.0, 1.0, 1.0, 1.0], 3) == [0, 1, 2, 4]
    assert contiguous_partition([3.0], 1) == [0, 1]
    with pytest.raises(ValueError):
        contiguous_partition([1.0], 2)
    rng = np.random.default_rng(0)
    for parts in (2, 3, 8):
        w = rng.uniform(1, 4, 256)
        b = contiguous_partition(w, parts)
        loads = [w[x:y].sum() for x, y in zip(b, b[1:])]
        assert max(loads) <= w.sum() / parts + w.max()


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the oracle arm prints from rank 0; the other ranks exit 0
    without work or output."""
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=_env(1, 2, _free_port()), capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""
