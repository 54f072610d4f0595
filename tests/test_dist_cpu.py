"""Multi-process paths of bench.py on CPU (gloo, world size 2).

Each GPU renders its own frame (replicas, no data-path collective); the only
exchange is the max of the timings over ranks, and the whole-job rate is the
sum of the ranks' queries over the slowest rank's time.  These tests run that
aggregation in two gloo processes, and the reference arm under torchrun, where
rank 0 alone prints its line.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=ws)
    import bench
    try:
        # rank r took (1 + r) ms on the device and (10 - r) ms end to end
        got = bench.reduce_max([1.0 + rank, 10.0 - rank], ws, "cpu")
        q.put((rank, bench._dist(), got))
    finally:
        dist.destroy_process_group()


def test_reduce_max_gloo_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [(2, 0, 0), (2, 1, 1)]
    for _, _, got in res:
        assert got == [2.0, 10.0]


def test_reduce_max_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max([3, 4.5], 1) == [3.0, 4.5]


def test_weak_throughput():
    sys.path.insert(0, ROOT)
    import bench
    # two replicas of a 1080p frame, slowest 0.25 ms: 2 * 2,073,600 / 0.25 ms
    assert bench.weak_throughput(2073600, 2, 0.25e-3) == pytest.approx(16.5888)
    assert bench.weak_throughput(2073600, 1, 0.25e-3) == pytest.approx(8.2944)


def test_reference_arm_under_torchrun_prints_once():
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
