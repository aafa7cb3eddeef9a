"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The single-instance path does not shard: with --gpus N every rank runs its own
replica and rank 0 reports the whole job from the max over ranks of the step
time (and the sum of the launch counts).  These tests run that logic as two
gloo processes on the host; no GPU is involved.
"""
from __future__ import annotations

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, q):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench

    r, lr, w = bench.dist_env()
    bench.rank_setup(lr, w, backend="gloo")
    mx = bench.over_ranks([r + 1.5, 10.0 - r], w, "max")
    sm = bench.over_ranks([r + 1.5, 10.0 - r], w, "sum")
    bench.rank_barrier(w)
    bench.rank_teardown(w)
    q.put((r, mx, sm))


def test_over_ranks_gloo_world2():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, mx, sm in out:
        assert mx == [2.5, 10.0]        # max over ranks of (1.5, 10) and (2.5, 9)
        assert sm == [4.0, 19.0]


def test_over_ranks_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.over_ranks([3, 4.5], 1, "max") == [3.0, 4.5]
    assert bench.over_ranks([3, 4.5], 1, "sum") == [3.0, 4.5]


def test_reference_arm_under_torchrun_world2():
    """The reference arm launched by torch.distributed.run with two ranks: rank 0 alone
    runs the oracle and prints one JSON line; the other rank exits 0."""
    pytest.importorskip("torch")
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
    assert d["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle"
