"""The multi-process path of bench.py on CPU: two gloo ranks agree on the
job time (the maximum over ranks) and the whole-job rate counts every
rank's replica; the reference arm runs on rank 0 only."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    mine = [10.0, 15.0][rank]
    t = bench.max_over_ranks(mine, world, device="cpu")
    rate = bench.whole_job_rate(1e9, world, t)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, rate))


def test_two_gloo_ranks_take_the_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[1] for g in got] == [15.0, 15.0]
    # 2 ranks x 1e9 units in 15 ms
    assert all(abs(g[2] - 2 * 1e9 / 15e-3 / 1e9) < 1e-9 for g in got)


def test_reference_arm_runs_on_rank0_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup = 1, 0
    assert bench.run_reference(A()) is None


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.whole_job_rate(5e8, 1, 1000.0) == 0.5
