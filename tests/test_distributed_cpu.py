"""The multi-process path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Every rank solves its own domain (weak scaling, no data-path collective); the
only collectives are the barrier and the max over ranks of the timed region.
"""
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
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2",
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist, r, ws, local = bench.dist_init(2)
    bench.barrier(dist)
    m = bench.max_over_ranks(dist, float(10 + rank))
    with open(os.path.join(out, f"rank{rank}.txt"), "w") as f:
        f.write(f"{r} {ws} {m}")
    dist.destroy_process_group()


def test_gloo_barrier_and_max_over_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        rank, ws, m = open(tmp_path / f"rank{r}.txt").read().split()
        assert int(rank) == r and int(ws) == 2 and float(m) == 11.0


def test_reference_arm_under_torchrun_two_ranks():
    """bench.py --impl reference launched like the driver does for N = 2: rank 0
    prints one JSON line, rank 1 exits 0 without work."""
    pytest.importorskip("torch")
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--boundary-nodes", "32",
           "--count", "8"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT,
                       env=dict(os.environ, OMP_NUM_THREADS="2"))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
