"""Multi-rank bench logic on CPU (gloo, world size 2): the timed value is the
whole-job throughput over the slowest rank, and only rank 0 reports.  The
GPU ranks run independent replicas, so no data-path collective is tested."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def max_over_ranks(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    local_ms = [40.0, 55.0][rank]  # rank 1 is the slowest
    ms, value = bench.job_throughput(local_ms, 4.0e10, world, max_over_ranks)
    dist.barrier()
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_two_rank_throughput_uses_slowest_rank():
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    for rank in (0, 1):
        ms, value = res[rank]
        assert ms == pytest.approx(55.0)
        assert value == pytest.approx(2 * 4.0e10 / 0.055 / 1e9)


def test_reference_arm_nonzero_rank_exits_quietly(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")

    class A:
        config = 1
        warmup = 0
        steps = 1
        gpus = 2

    bench.run_reference(A())
    assert capsys.readouterr().out == ""
