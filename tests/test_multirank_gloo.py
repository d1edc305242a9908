"""The multi-rank logic of bench.py on CPU ranks (gloo, world size 2): the
barrier, the max over ranks of the per-step time and the whole-job value.
Replicas run independent problems, so no data-path collective exists."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    assert bench.dist_env() == (ws, rank, rank)
    bench.barrier(ws)
    local_ms = 10.0 + 5.0 * rank           # rank 1 is the slower replica
    ms = bench.max_over_ranks(ws, local_ms)
    q.put((rank, ms, bench.job_value(ws, ms)))
    bench.barrier(ws)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(ws))
    for rank, ms, value in out:
        assert ms == 15.0                   # max over ranks
        assert value == pytest.approx(2 * 1000.0 / 15.0)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(1, 7.0) == 7.0
    assert bench.job_value(1, 10.0) == 100.0


def test_bench_spawns_one_rank_per_gpu_without_torchrun():
    """bench.py --gpus N started without WORLD_SIZE re-launches itself under
    torch.distributed.run with N local ranks, the same arguments and a
    127.0.0.1 rendezvous."""
    import sys

    import bench
    cmd = bench.spawn_command(["--gpus", "4", "--steps", "5"], 4, 29512)
    assert cmd[:3] == [sys.executable, "-m", "torch.distributed.run"]
    i = cmd.index("--nproc-per-node")
    assert cmd[i + 1] == "4"
    assert cmd[cmd.index("--master-addr") + 1] == "127.0.0.1"
    assert cmd[cmd.index("--master-port") + 1] == "29512"
    assert cmd[-5].endswith("bench.py") and cmd[-4:] == ["--gpus", "4", "--steps", "5"]
