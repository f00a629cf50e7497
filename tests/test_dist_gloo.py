"""Multi-rank host logic of bench.py on CPU: two gloo ranks, as torchrun
would launch them on two GPUs.  Each rank prices its own replica (distinct
digital shift), the timing is the maximum over ranks, and the reference arm
runs on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads
    opt = bench.replica_option(workloads.single_large(), rank)
    t_ms = 10.0 + 3.0 * rank                         # rank 1 is the slow one
    t_max = bench.max_over_ranks(dist, t_ms)
    value = opt.path_steps * world / (t_max * 1e-3)
    q.put((rank, opt.seed, t_max, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max_timing():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, s0, t0, v0), (_, s1, t1, v1) = out
    assert s0 != s1 and {s0, s1} == {2, 3}
    assert t0 == t1 == 13.0
    assert v0 == v1 == pytest.approx(2 * 252 * 2 ** 20 / 13e-3)


def test_reference_arm_rank_nonzero_exits_without_work(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        gpus, steps, warmup = 2, 1, 3
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
