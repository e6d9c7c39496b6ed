"""The multi-rank bench path on CPU: two gloo ranks (127.0.0.1) agree on the slowest rank's
time, the whole-job rate counts every rank's work, and only rank 0 runs the oracle arm."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank                     # rank 1 is the slow one
    mx = bench.max_over_ranks(ms, world)
    out.put((rank, mx, bench.job_rate(40, world, mx)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [150.0, 150.0]
    # 2 ranks x 40 units in 0.15 s
    assert res[0][2] == pytest.approx(2 * 40 / 0.15)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_rate(10, 1, 500.0) == pytest.approx(20.0)


def test_reference_arm_runs_on_rank_0_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        workload, steps, warmup, gpus = "plain_32", 1, 0, 2
    assert bench.run_reference(A()) is None
    assert capsys.readouterr().out == ""
