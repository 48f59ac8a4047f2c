"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas only, no
data-path collective), max-over-ranks timing and the whole-job rate, and the
reference arm's rank > 0 exiting without work."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        t = bench.max_over_ranks(times[rank], dist, device="cpu")
        out[rank] = (t, bench.whole_job_rate(world, 16 * 5, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    world = 2
    times = [2.0, 3.0]
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, times, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    t, rate = res[0]
    assert t == 3.0
    assert rate == pytest.approx(world * 16 * 5 / 3.0)


def test_single_rank_is_identity():
    assert bench.max_over_ranks(1.25, None) == 1.25
    assert bench.whole_job_rate(1, 80, 2.0) == 40.0


def test_reference_arm_other_ranks_do_no_work(capsys):
    class A:
        steps = 1
        warmup = 0
        gpus = 2

    assert bench.run_reference(A(), rank=1, world=2) is None
    assert capsys.readouterr().out == ""
