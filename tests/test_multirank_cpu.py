"""The benchmark's multi-rank arithmetic under torch.distributed with the gloo backend on CPU
(two ranks): the timed region is the slowest rank's, and the job rate counts every rank's
evaluations. The GPU path itself is replicas (one bunch per rank, no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
    t = bench.max_over_ranks(ms, world, device="cpu")
    out[rank] = (t, bench.job_rate(8, world, t))
    torch.distributed.barrier()
    torch.distributed.destroy_process_group()


def test_two_rank_timing_is_max_and_rate_counts_all_ranks():
    world = 2
    port = _free_port()
    # the manager's server process spawned too: no fork of a process that may hold threads
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert res[0][1] == pytest.approx(8 * 2 / 0.015)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_rate(10, 1, 20.0) == pytest.approx(500.0)
