"""The N > 1 path of bench.py on the CPU: N independent replicas (one problem per rank,
no collective on the data path) that meet at barriers and in the max of their times,
run here as two gloo ranks; and the reference arm's rank rule (rank 0 alone works)."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r = bench.Replicas(world, "cpu", dist)
    r.barrier()
    ms = r.max(10.0 + 5.0 * rank)          # rank times 10 and 15 ms
    rate = r.rate(1000, 4, ms)             # 1000 units per rank and step, 4 steps
    r.barrier()
    out.put((rank, ms, rate))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_sum_the_work():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in got:
        assert ms == 15.0                          # the max over ranks, on every rank
        assert rate == pytest.approx(2 * 1000 * 4 / 0.015)   # both ranks' units


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Replicas(1, "cpu")
    r.barrier()
    assert r.max(3.5) == 3.5
    assert r.rate(10, 2, 4.0) == pytest.approx(10 * 2 / 0.004)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0 and p.stdout.strip() == ""
