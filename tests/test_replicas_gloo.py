"""Multi-GPU form of the bench is independent replicas (a single solve does
not shard without a per-stage panel exchange): each rank times its own solve
and the job reports all ranks' work over the slowest rank's time.  The rank
aggregation is exercised here with world_size 2 on the gloo backend (CPU)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    slowest = bench.max_over_ranks(100.0 + 50.0 * rank, "cpu")  # rank 1 is the slow one
    q.put((rank, slowest, bench.job_value(10.0, world, slowest)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_with_gloo():
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
    assert [r[1] for r in res] == [150.0, 150.0]
    assert all(r[2] == pytest.approx(2 * 10.0 / 150.0) for r in res)


def test_reference_arm_other_ranks_exit_quietly(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        dtype, n, steps, warmup, gpus = "f32", 16384, 1, 0, 2
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
