"""The bench's multi-rank logic on CPU: two gloo ranks (world size 2) time
different amounts of work; the reported time is the slowest rank's and the
throughput counts the units of both ranks.  The reference arm under torchrun
prints one line, from rank 0, and every rank exits 0."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist = bench.dist_init(world, "gloo")
    bench.barrier(world)
    rank_ms = 100.0 * (rank + 1)                      # rank 1 is the slow one
    value, total_ms = bench.whole_job_throughput(1e6, 10, rank_ms, world)
    out.put((rank, value, total_ms, bench.reduce_max(float(rank), world)))
    bench.barrier(world)
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_whole_job_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, total_ms, rmax in res:
        assert total_ms == 200.0                       # the slowest rank
        assert value == pytest.approx(2 * 1e6 * 10 / 0.2)
        assert rmax == 1.0


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    value, total_ms = bench.whole_job_throughput(5.0, 4, 20.0, 1)
    assert total_ms == 20.0 and value == pytest.approx(5.0 * 4 / 0.02)


def test_reference_arm_under_torchrun_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--ref-sample", "300"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300,
                       env={**os.environ, "ORACLE_THREADS": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
