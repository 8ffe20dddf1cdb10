"""The multi-rank bookkeeping of bench.py on CPU ranks (gloo, world size 2): the
whole-job time is the maximum over ranks and the throughput counts every rank's
units; the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 40.0][rank]
    total = bench.max_over_ranks(ms, dist, "cpu")
    out[rank] = (total, bench.job_throughput(1000.0, world, total))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        total, value = res[rank]
        assert total == 40.0                        # the slowest rank sets the job time
        assert value == pytest.approx(2 * 1000.0 / 0.040)
    assert bench.max_over_ranks(7.0) == 7.0
    assert bench.job_throughput(10.0, 1, 1000.0) == pytest.approx(10.0)


def test_reference_arm_runs_on_rank0_only(capsys):
    class A:
        steps, warmup = 1, 0
    bench.run_reference(A(), world=2, rank=1)      # a non-zero rank returns without work
    assert capsys.readouterr().out == ""
