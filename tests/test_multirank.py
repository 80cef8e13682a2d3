"""Replicas across ranks (world_size 2, gloo, CPU): each rank reduces its own
invocation -- no data-path collective -- and the job's time is the slowest
rank's. Runs the same helpers bench.py uses, with the oracle standing in for
the GPU reduction so that no device is needed."""
from __future__ import annotations

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    import synth
    tr = synth.large(seed=rank, n_mem=20_000, n_br=5_000, n_wi=8, per_wi=200, zipf_distinct=1 << 12)
    m = oracle.compute(tr)
    seconds = 0.5 + rank  # rank 1 is the slowest replica
    slowest = bench.max_over_ranks(seconds, dist, "cpu")
    value = bench.replica_throughput(tr.n_mem, world, slowest)
    # no data-path exchange: gather the per-rank results only to check them here
    got = [None] * world
    dist.all_gather_object(got, (m["footprint"], m["entropy"][0], value))
    if rank == 0:
        out.put(got)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_slowest_rank_sets_the_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (fp0, h0, v0), (fp1, h1, v1) = got
    assert v0 == v1 == pytest.approx(2 * 20_000 / 1.5)  # 2 replicas x 20,000 events / slowest 1.5 s
    assert (fp0, h0) != (fp1, h1)  # replicas reduce different invocations (seed = rank)


def _leaving_rank(rank, world, port, out):
    """Rank 1 fails between steps (it exits before the timing reduction); rank
    0 must get an error from that reduction, not wait for ever."""
    from datetime import timedelta
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=10))
    import bench
    if rank == 1:
        os._exit(3)  # a replica that dies with no collective in flight
    try:
        bench.max_over_ranks(1.0, dist, "cpu")
        out.put("no error")
    except Exception as e:  # gloo: connection closed by the peer, or the timeout
        out.put(type(e).__name__)
    out.close()
    out.join_thread()
    os._exit(0)  # skip process-group teardown with a dead peer


def test_a_rank_that_leaves_fails_the_others_collective():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_leaving_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert got in ("RuntimeError", "DistBackendError", "DistError", "DistNetworkError"), got
    assert procs[1].exitcode == 3 and procs[0].exitcode == 0
