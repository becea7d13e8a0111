"""bench.py's multi-rank logic on the CPU (gloo, two ranks): the ranks meet at
the barrier and agree on the maximum of their timings, which is what the
replicated GPU run reports; the reference arm does its work on rank 0 only."""
import json
import os
import socket
import subprocess
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]

RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import bench
ctx = bench.Ctx(cpu=True)
ctx.barrier()
m = ctx.max_over_ranks(1.5 + ctx.rank)
ctx.barrier()
ctx.close()
print(json.dumps({{"rank": ctx.rank, "world": ctx.world, "max": m}}))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_agree_on_max_time():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_SCRIPT.format(root=str(ROOT))], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=300) for p in procs]
    for p, (out, err) in zip(procs, outs):
        assert p.returncode == 0, err[-2000:]
    got = sorted((json.loads(o.strip().splitlines()[-1]) for o, _ in outs), key=lambda d: d["rank"])
    assert [d["rank"] for d in got] == [0, 1] and all(d["world"] == 2 for d in got)
    assert all(d["max"] == 2.5 for d in got)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "conv", "--steps", "1",
                          "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""
