"""bench.py's multi-rank timing on the CPU (gloo, world size 2): the barrier returns on
both ranks and max_over_ranks gives every rank the largest of the ranks' values, which is
what the replicas' timing takes (whole-job value = units of all ranks / the slowest rank's
time).  A world of one needs no process group."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SNIPPET = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import torch, bench
rank, world, barrier, max_over_ranks = bench.rank_context(torch, "cpu")
barrier()
m = max_over_ranks(1.5 + rank)
barrier()
import torch.distributed as dist
dist.destroy_process_group()
print(json.dumps({{"rank": rank, "world": world, "max": m}}))
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_gloo():
    pytest.importorskip("torch")
    port = free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", SNIPPET.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=300)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    assert all(o["world"] == 2 and o["max"] == 2.5 for o in outs)


def test_world_of_one():
    torch = pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.pop(k) for k in ("RANK", "WORLD_SIZE") if k in os.environ}
    try:
        rank, world, barrier, max_over_ranks = bench.rank_context(torch, "cpu")
        barrier()
        assert (rank, world, max_over_ranks(3.25)) == (0, 1, 3.25)
    finally:
        os.environ.update(env)
