"""The N > 1 launch path of bench.py on CPU: two ranks over gloo.

Solves are independent problems (replicas, weak scaling), so the only
collectives are the barrier and the max / sum over ranks of the timing;
these tests run them with world size 2 on the host, and run the reference
arm under torchrun with two ranks (rank 0 alone measures and prints)."""
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
    port = s.getsockname()[1]
    s.close()
    return port


_WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import bench
D = bench.Dist(want_cuda=False)
out = dict(rank=D.rank, world=D.world, mx=D.max(float(D.rank) + 0.5), sm=D.sum(D.rank + 1))
D.barrier()
D.close()
print(json.dumps(out), flush=True)
"""


def test_dist_collectives_two_ranks_gloo():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", _WORKER.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for o in outs:
        assert o["world"] == 2
        assert o["mx"] == 1.5           # max over ranks of rank + 0.5
        assert o["sm"] == 3.0           # 1 + 2
    assert sorted(o["rank"] for o in outs) == [0, 1]


def test_reference_arm_two_ranks_prints_one_line():
    pytest.importorskip("torch")
    port = _free_port()
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--cpu-seconds", "1"]
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, p.stdout
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["value"] > 0
    assert out["e2e"]["h2d_bytes_per_step"] == 0
    assert out["cpu_baseline"]["kind"] == "oracle"
