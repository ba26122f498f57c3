"""The multi-GPU path of the benchmark on the host: N independent replicas
(the step has no data exchange between GPUs), a barrier around each timed
region and the max over ranks of its duration.  Two gloo ranks on the CPU,
each a separate process with the environment torchrun would give it."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["REPO_ROOT"])
import bench
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
r = bench.Replicas(world, backend="gloo")
r.barrier()
t = [0.010, 0.030][rank]                       # this rank's timed region, seconds
out = {"max": r.max(t), "value": r.throughput(100.0, t)}
r.barrier()
r.close()
print(json.dumps(out))
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def run_ranks(world=2, timeout=120):
    port = free_port()
    procs = []
    for rank in range(world):
        env = dict(os.environ, REPO_ROOT=ROOT, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        so, se = p.communicate(timeout=timeout)
        assert p.returncode == 0, se
        outs.append(json.loads(so.strip().splitlines()[-1]))
    return outs


def test_replicas_report_the_slowest_rank_and_the_whole_job():
    r0, r1 = run_ranks()
    assert r0["max"] == r1["max"] == 0.030                   # max over ranks, seen by every rank
    assert abs(r0["value"] - 2 * 100.0 / 0.030) < 1e-9       # all ranks' units over the slowest time
    assert r0["value"] == r1["value"]


def test_single_process_needs_no_process_group():
    import bench
    r = bench.Replicas(1)
    assert r.dist is None and r.max(0.5) == 0.5 and r.throughput(10.0, 0.5) == 20.0
    r.barrier()
    r.close()


def test_reference_arm_prints_on_rank_zero_only(capsys):
    import argparse
    import bench
    assert bench.run_reference(argparse.Namespace(), world=2, rank=1) == 0
    assert capsys.readouterr().out == ""
