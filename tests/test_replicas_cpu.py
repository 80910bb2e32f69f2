"""The N > 1 path of the bench (independent replicas, no data-path collective),
run as two gloo ranks on the CPU: the barrier, the max over ranks, the
whole-job throughput, and the reference arm printing on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

from conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    bench._barrier(ws)
    slowest = bench._max_over_ranks(ws, 1.0 + rank)          # rank 1 is the slow one
    value = bench.replica_throughput(ws, 1000, 10, 1.0 + rank)
    q.put((rank, slowest, value))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, value in out:
        assert slowest == 2.0
        assert value == pytest.approx(2 * 1000 * 10 / 2.0)


def test_reference_arm_prints_on_rank_zero_only():
    # under torchrun the reference arm runs on rank 0; other ranks exit 0 silently
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip() == ""
