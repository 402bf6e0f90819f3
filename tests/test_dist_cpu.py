"""The multi-rank host logic of the bench on CPU: two gloo ranks (replicas
of the workload) agree on the step time (the maximum over ranks) and on
the whole-job throughput, which counts every rank's DOF."""
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


def _rank(rank, world, port, out):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = 0.010 + 0.005 * rank          # seconds per step on this rank
        t = bench.max_over_ranks(local, world)
        out.put((rank, t, bench.job_gdofs(world, 1_000_000, t)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_reduce_the_step_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    times = {r: t for r, t, _ in res}
    rates = {r: v for r, _, v in res}
    assert times[0] == times[1] == pytest.approx(0.015)
    # 2 replicas x 1e6 DOF x 4 RHS per step / 15 ms
    assert rates[0] == rates[1] == pytest.approx(2 * 1e6 * 4 / 0.015 / 1e9)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(0.02, 1) == 0.02
    assert bench.job_gdofs(1, 42_390_000, 0.149) == pytest.approx(42.39e6 * 4 / 0.149 / 1e9)
