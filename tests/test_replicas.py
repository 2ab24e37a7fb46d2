"""CPU checks of the N > 1 path of bench.py: one replica solve per rank, no
collective on the data path, the job's time taken as the slowest rank's.  Two
gloo ranks on 127.0.0.1 stand in for two GPUs; a rank that fails before the
timing barrier is seen by the other on the host, as an error, not a hang."""
import datetime
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))


def _timing_rank(rank, world, port, out):
    _init(rank, world, port)
    dist.barrier()
    elapsed = [2.0, 5.0][rank]  # the second rank is slower
    t = bench.max_over_ranks(elapsed, dist, "cpu")
    out[rank] = (t, bench.job_rate(10, world, t))
    dist.barrier()
    dist.destroy_process_group()


def _failing_rank(rank, world, port, out):
    _init(rank, world, port)
    if rank == 1:
        raise SystemExit(3)  # leaves before the timing barrier, with nothing in flight
    try:
        dist.barrier()
        out[rank] = "no error"
    except Exception as e:  # the peer is gone: the collective ends with an error
        out[rank] = type(e).__name__


def test_job_time_is_the_slowest_rank_and_value_counts_all_ranks():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_timing_rank, args=(2, _port(), out), nprocs=2, join=True, start_method="spawn")
    assert out[0] == out[1] == (5.0, 2 * 10 / 5.0)


def test_single_rank_needs_no_collective():
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_rate(10, 1, 2.0) == 5.0


def test_a_rank_that_leaves_is_seen_by_the_other_as_an_error():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    ctx = mp.start_processes(_failing_rank, args=(2, _port(), out), nprocs=2, join=False, start_method="spawn")
    for p in ctx.processes:
        p.join(timeout=60)
    codes = [p.exitcode for p in ctx.processes]
    assert codes[1] == 3
    assert out.get(0) not in (None, "no error"), out
