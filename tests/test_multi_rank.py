"""Host logic of `bench.py --gpus N` (N > 1) on CPU: world-size-2 gloo ranks.

With N GPUs the bench runs N independent replicas of the workload (the path
has no exchange step, so no collective touches the data path).  What needs
checking without GPUs is the timing aggregation: the step time is the maximum
over ranks, the whole-job value counts every rank's group, and the reference
arm runs on rank 0 only.
"""
import importlib.util
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        local = [12.5, 40.25][rank]  # ms per step seen by this rank
        t = b.max_over_ranks(local)
        dist.barrier()
        out[rank] = (t, b.job_value(world, t), b.dist_env()[:2])
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo_world2():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        t, v, env = res[rank]
        assert t == 40.25  # every rank gets the slowest rank's time
        assert v == pytest.approx(2 * 1000.0 / 40.25)  # two groups per step
        assert env == (2, rank)


def test_single_process_aggregation_is_identity():
    b = _bench()
    assert b.max_over_ranks(3.5) == 3.5
    assert b.job_value(1, 50.0) == pytest.approx(20.0)


def test_reference_arm_runs_on_rank0_only(monkeypatch, capsys):
    b = _bench()
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class A:
        scale, k, steps, warmup = 10, 2, 1, 0

    assert b.run_reference(A()) is None  # returns before any work
    assert capsys.readouterr().out == ""
