"""Host-side multi-rank logic of bench.py on CPU (gloo, world size 2): the path
shards into independent replicas (weak scaling, no data-path collective); the
only collectives are the barrier and the max-over-ranks of the timings."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [120.0, 180.0][rank]
    ms = bench.reduce_max(ms_local, dist, torch.device("cpu"))
    dist.barrier()
    v = bench.job_throughput(1000, 10, 2, world, ms)
    # every rank draws its own seeded replica
    case = bench.workload("adjoint128", rank, 1)
    out[rank] = (ms, v, int(case.labels.sum()))
    dist.destroy_process_group()


def test_two_ranks_max_time_and_whole_job_throughput():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 180.0
    assert res[0][1] == res[1][1] == pytest.approx(1000 * 10 * 2 * 2 / 0.18 / 1e9)
    assert res[0][2] != res[1][2]                 # different seeded phantoms per rank


def test_single_process_is_identity():
    assert bench.reduce_max(3.5, None, torch.device("cpu")) == 3.5
    assert bench.job_throughput(100, 10, 1, 1, 1.0) == pytest.approx(1e-3)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    args = bench.parse_args(["--impl", "reference", "--gpus", "2"])
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
