"""Sharded invocations through the C ABI on the GPU: ranks route their slices,
exchange them, reduce their shards with the finalisation deferred and export
their exact distributions; merging the blobs must give the whole invocation's
metrics bit for bit -- equal to one device reducing it alone, and to the
oracle. Ranks are emulated in one process (the all-to-all is a list
transpose) and, separately, run as two gloo processes sharing the GPU (their
kernels never wait on one another; only host buffers are exchanged)."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch

import oracle
import synth
from tests.helpers import random_trace
from tests.test_gpu_parity import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_04207_gb300 as P
    return P


def _slices(S, whole, world):
    """Contiguous per-rank slices of every stream (push order across ranks)."""
    out = []
    for r in range(world):
        def part(a, unit):
            n = a.size // unit
            return a[unit * (r * n // world):unit * ((r + 1) * n // world)]
        R = whole.run_wi.size
        lo, hi = r * R // world, (r + 1) * R // world
        out.append(S.Slice(part(whole.mem, 16), part(whole.br, 8), whole.run_wi[lo:hi], whole.run_off[lo:hi],
                           whole.run_len[lo:hi], whole.ops,
                           part(whole.widths.view(np.uint8), 2).view(np.uint16)))
    return out


def _sharded(P, tr, world, **cfg):
    from paper_1805_04207_gb300 import shard as S
    from paper_1805_04207_gb300.api import Characterizer
    cfg.setdefault("n_opcodes", tr.n_opcodes)
    whole = S.Slice.of_trace(tr)
    mine = _slices(S, whole, world)
    routed = [S.route(m, world, cfg.get("byte_addresses", 0)) for m in mine]
    blobs = []
    for r in range(world):
        with Characterizer(**cfg) as c:
            for src in range(world):  # the all-to-all: shard r of every rank, in source-rank order
                S.push_slice(c, routed[src][r])
            if mine[r].widths.size:
                c.push_widths(mine[r].widths)
            blobs.append(P.aiwc_shard_export(c.h))
    with Characterizer(**cfg) as c:
        hist = np.zeros(tr.n_opcodes, dtype=np.uint64)
        out = P.aiwc_shard_merge(c.h, blobs, hist)
        out["opcode_hist"] = hist
    return out


def _single(P, tr, **cfg):
    from paper_1805_04207_gb300.api import Characterizer, push_trace
    cfg.setdefault("n_opcodes", tr.n_opcodes)
    with Characterizer(**cfg) as c:
        push_trace(c, tr.to("cuda"))
        return c.compute()


def _identical(a, b):
    for k, v in b.items():
        if k == "opcode_hist":
            assert np.array_equal(np.asarray(a[k]), np.asarray(v)), k
        elif isinstance(v, float) and np.isnan(v):
            assert np.isnan(a[k]), k
        else:
            assert a[k] == v, (k, a[k], v)


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_sharded_large_shape_equals_one_device_and_oracle(P, world):
    tr = synth.large(seed=7, n_mem=400_003, n_br=120_001, n_wi=300, per_wi=999, zipf_distinct=1 << 16)
    g = _sharded(P, tr, world)
    assert_parity(g, oracle.compute(tr))
    _identical(g, _single(P, tr))


@pytest.mark.parametrize("opts", [dict(plan=1), dict(history_scope=1, history_len=5), dict(byte_addresses=1),
                                  dict(space_mask=0x5, precision=1)])
def test_sharded_options(P, opts):
    tr = random_trace(31, n_mem=3000, n_br=2500, n_wi=9, n_runs=50, n_ops=4000, addr_pool=700, n_sites=6,
                      addr_span_bits=14, size_choices=[1, 2, 4, 8] if opts.get("byte_addresses") else None)
    g = _sharded(P, tr, 3, **opts)
    ocfg = {k: v for k, v in opts.items() if k in ("history_scope", "history_len", "byte_addresses", "space_mask")}
    assert_parity(g, oracle.compute(tr, **ocfg), entropy_tol=2.0 ** -22 if opts.get("precision") else 1e-9)
    _identical(g, _single(P, tr, **opts))


def test_tiny_workload_sharded(P):
    tr = synth.tiny()
    _identical(_sharded(P, tr, 2), _single(P, tr))


def test_merge_checks_its_blobs(P):
    from paper_1805_04207_gb300.api import Characterizer
    tr = random_trace(2, n_mem=100, n_br=100, n_runs=4, n_ops=80)
    with Characterizer(n_opcodes=tr.n_opcodes) as c:
        c.push_mem(tr.mem.cuda())
        blob = P.aiwc_shard_export(c.h)
        # the handle is free again for the next invocation
        c.push_mem(tr.mem.cuda())
        c.compute()
    with Characterizer(n_opcodes=tr.n_opcodes, history_len=7) as c:  # another metric configuration
        with pytest.raises(P.AiwcError) as e:
            P.aiwc_shard_merge(c.h, [blob])
        assert e.value.status == P.AIWC_EINVAL
    with Characterizer(n_opcodes=tr.n_opcodes) as c:
        with pytest.raises(P.AiwcError) as e:
            P.aiwc_shard_merge(c.h, [blob[:-8]])
        assert e.value.status == P.AIWC_EINVAL
        c.push_mem(tr.mem.cuda())
        with pytest.raises(P.AiwcError) as e:
            P.aiwc_shard_merge(c.h, [blob])  # pushed events of another invocation pending
        assert e.value.status == P.AIWC_ESTATE
        c.compute()
        # the same blob twice is two ranks that each saw these events: counts double
        d = P.aiwc_shard_merge(c.h, [blob, blob])
        assert d["total_reads"] + d["total_writes"] == 2 * tr.n_mem
    with Characterizer(n_opcodes=tr.n_opcodes, partitions=2) as c:
        with pytest.raises(P.AiwcError) as e:
            P.aiwc_shard_export(c.h)
        assert e.value.status == P.AIWC_EINVAL


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _proc_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=__import__("datetime").timedelta(seconds=120))
    from paper_1805_04207_gb300 import shard as S
    from paper_1805_04207_gb300.api import Characterizer
    tr = synth.large(seed=9, n_mem=200_001, n_br=50_001, n_wi=100, per_wi=777, zipf_distinct=1 << 14)
    whole = S.Slice.of_trace(tr)
    mine = _slices(S, whole, world)[rank]
    with Characterizer(device=0, n_opcodes=tr.n_opcodes) as c:
        out = S.reduce_sharded(c, mine)
    got = [None] * world
    dist.all_gather_object(got, {k: (v.tolist() if isinstance(v, np.ndarray) else v) for k, v in out.items()})
    if rank == 0:
        q.put(got)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_on_one_gpu(P):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_proc_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    import json
    assert json.dumps(got[0], sort_keys=True) == json.dumps(got[1], sort_keys=True)  # both hold the whole result
    tr = synth.large(seed=9, n_mem=200_001, n_br=50_001, n_wi=100, per_wi=777, zipf_distinct=1 << 14)
    g = dict(got[0])
    g["opcode_hist"] = np.asarray(g["opcode_hist"], dtype=np.uint64)
    assert_parity(g, oracle.compute(tr))
