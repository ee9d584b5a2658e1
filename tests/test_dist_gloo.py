"""The multi-rank path of bench.py on CPU.  Two gloo ranks, started the way
torchrun starts them (one process per rank, RANK / WORLD_SIZE / MASTER_ADDR /
MASTER_PORT in the environment), each time their own replica, so the job's
step time is the maximum over ranks: one all-reduce of a scalar.  The
reference arm does its work and prints on rank 0 only; other ranks exit
without output."""
import json
import os
import socket
import subprocess
import sys

import pytest

pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import contextlib, io, json, os, sys
sys.path.insert(0, os.environ["MAHI_ROOT"])
import bench
dist, rank, ws = bench._dist()
step_ms = bench._max_over_ranks(dist, 1.5 + rank, "cpu")
out = io.StringIO()
if rank != 0:
    with contextlib.redirect_stdout(out):
        bench.run_reference(None)
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "ws": ws, "step_ms": step_ms, "reference_output": out.getvalue()}))
"""


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_take_the_max_and_only_rank0_reports():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), MAHI_BENCH_GLOO="1", MAHI_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    try:
        outs = [p.communicate(timeout=180) for p in procs]
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    for p, (_, err) in zip(procs, outs):
        assert p.returncode == 0, err[-2000:]
    recs = sorted((json.loads(o.strip().splitlines()[-1]) for o, _ in outs), key=lambda d: d["rank"])
    assert [d["rank"] for d in recs] == [0, 1]
    assert all(d["ws"] == 2 for d in recs)
    assert all(d["step_ms"] == 2.5 for d in recs)  # max(1.5, 2.5) on both ranks
    assert recs[1]["reference_output"] == ""
