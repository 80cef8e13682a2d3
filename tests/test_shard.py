"""Sharded invocations on the CPU: the library's routing keeps every unit of
the method whole, and a world_size-2 gloo job (route, all-to-all, per-rank
reduction, sum) reproduces the whole invocation's exact distributions.

Without a GPU the per-rank reduction is the oracle's: the distributions a
rank exports (count-of-counts per skip level, pattern and ITB counts, totals)
are what the oracle computes on the rank's shard, and their sum over ranks
must be the oracle's on the whole trace (Sec. V adds work-groups' results
into global state; the partition pins show the sum is exact for whole units).
"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from tests.helpers import random_trace


def _P():
    import paper_1805_04207_gb300 as P
    return P


def _shard_mod():
    from paper_1805_04207_gb300 import shard
    return shard


def _sb_keys(mem_u8):
    ev = mem_u8.reshape(-1, 16)
    addr = ev[:, :8].copy().view(np.uint64).reshape(-1)
    space = (ev[:, 13] >> 1) & 3
    return (space.astype(np.uint64) << np.uint64(56)) | ((addr & np.uint64((1 << 61) - 1)) >> np.uint64(11))


@pytest.mark.parametrize("n_shards", [1, 2, 3, 8])
def test_memory_routing_keeps_superblocks_whole_and_order(n_shards):
    S = _shard_mod()
    tr = synth.large(seed=5, n_mem=30_000, n_br=0, n_wi=0, per_wi=1, zipf_distinct=1 << 14)
    sl = S.Slice.of_trace(tr)
    shards = S.route(sl, n_shards)
    assert sum(s.mem.size for s in shards) == sl.mem.size
    seen = {}
    for k, s in enumerate(shards):
        for key in np.unique(_sb_keys(s.mem)):
            assert seen.setdefault(int(key), k) == k  # a superblock lives in one shard
    # stable: each shard is the input's subsequence of its superblocks
    rec = sl.mem.reshape(-1, 16)
    keys = _sb_keys(sl.mem)
    owner = np.array([seen[int(x)] for x in keys])
    for k, s in enumerate(shards):
        assert np.array_equal(s.mem.reshape(-1, 16), rec[owner == k])


def test_byte_routing_splits_accesses_at_superblock_edges():
    P = _P()
    from tests.helpers import mem_only
    tr = mem_only([2046, 100, 4094], sizes=[4, 8, 2])  # the first crosses 2048, the last ends at 4095
    routed, counts = P.aiwc_shard_route_mem(2, tr.mem.numpy(), byte_addresses=1)
    ev = routed.reshape(-1, 16)
    assert ev.shape[0] == 4 and int(counts.sum()) == 4
    got = sorted((int(e[:8].view(np.uint64)[0]), int(e[12])) for e in ev)
    assert got == [(100, 8), (2046, 2), (2048, 2), (4094, 2)]
    # without byte addresses nothing is split
    routed, counts = P.aiwc_shard_route_mem(2, tr.mem.numpy(), byte_addresses=0)
    assert routed.size == 48 and int(counts.sum()) == 3


def test_branch_and_run_routing_keep_sites_and_work_items_whole():
    S = _shard_mod()
    tr = random_trace(3, n_mem=0, n_br=500, n_wi=7, n_runs=40, n_ops=900, n_sites=9)
    sl = S.Slice.of_trace(tr)
    shards = S.route(sl, 3)
    sites = [set(np.frombuffer(s.br.tobytes(), np.uint32)[0::2].tolist()) for s in shards]
    assert all(not (a & b) for i, a in enumerate(sites) for b in sites[i + 1:])
    assert sum(s.br.size for s in shards) == sl.br.size
    wis = [set(s.run_wi.tolist()) for s in shards]
    assert all(not (a & b) for i, a in enumerate(wis) for b in wis[i + 1:])
    # every run keeps its opcodes, and a shard's offsets index its own segment
    orig = {}
    for w, o, ln in zip(sl.run_wi, sl.run_off, sl.run_len):
        orig.setdefault(int(w), []).append(sl.ops[int(o):int(o) + int(ln)].tolist())
    for s in shards:
        got = {}
        for w, o, ln in zip(s.run_wi, s.run_off, s.run_len):
            got.setdefault(int(w), []).append(s.ops[int(o):int(o) + int(ln)].tolist())
        for w, runs in got.items():
            assert runs == orig[w]  # same runs, same order


def test_routing_rejects_bad_arguments():
    P = _P()
    with pytest.raises(P.AiwcError):
        P.aiwc_shard_route_branch(0, np.zeros(8, np.uint8))
    with pytest.raises(P.AiwcError):
        P.aiwc_shard_route_runs(2, [0], [5], [10], np.zeros(8, np.uint16))  # run past its opcodes


def test_slice_pack_round_trip():
    S = _shard_mod()
    sl = S.Slice.of_trace(random_trace(4, n_mem=30, n_br=20, n_runs=5, n_ops=50))
    back = S.Slice.unpack(sl.pack())
    for f in ("mem", "br", "run_wi", "run_off", "run_len", "ops"):
        assert np.array_equal(getattr(back, f), getattr(sl, f)), f


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _distributions(tr, h=16):
    """What a rank exports, computed by the oracle: count-of-counts of every
    skip level and the integer totals that add over whole units."""
    o = oracle.compute(tr, history_len=h)
    coc = [oracle.count_of_counts(tr.mem, n) if tr.mem is not None and tr.mem.shape[0] else {} for n in range(11)]
    ints = [o[k] for k in ("total_reads", "total_writes", "footprint", "unique_reads", "unique_writes",
                           "branch_events", "branch_sites", "branch_patterns", "branch_minsum", "barriers",
                           "itb_count", "ipt_count", "total_instructions")]
    return coc, ints, np.asarray(o["opcode_hist"], dtype=np.uint64)


def _trace_of(sl, n_opcodes):
    t = synth.Trace("shard", mem=torch.from_numpy(sl.mem.copy()).view(torch.int64).reshape(-1, 2),
                    br=torch.from_numpy(sl.br.copy()).view(torch.int64),
                    ops=torch.from_numpy(sl.ops.astype(np.int16)),
                    run_wi=torch.from_numpy(sl.run_wi.astype(np.int64)),
                    run_off=torch.from_numpy(sl.run_off.astype(np.int64)),
                    run_len=torch.from_numpy(sl.run_len.astype(np.int64)), n_opcodes=n_opcodes)
    return t


def _gloo_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1805_04207_gb300 import shard as S
    tr = random_trace(11, n_mem=4000, n_br=3000, n_wi=6, n_runs=60, n_ops=5000, addr_pool=900, n_sites=7,
                      addr_span_bits=16)
    whole = S.Slice.of_trace(tr)
    # this rank's contiguous slice of every stream (push order kept across ranks)
    def part(a, unit):
        n = a.size // unit
        lo, hi = rank * n // world, (rank + 1) * n // world
        return a[unit * lo:unit * hi]
    R = whole.run_wi.size
    lo, hi = rank * R // world, (rank + 1) * R // world
    mine = S.Slice(part(whole.mem, 16), part(whole.br, 8), whole.run_wi[lo:hi], whole.run_off[lo:hi],
                   whole.run_len[lo:hi], whole.ops)
    got = S.exchange(S.route(mine, world), None)
    mine_all = S.Slice(np.concatenate([g.mem for g in got]), np.concatenate([g.br for g in got]),
                       np.concatenate([g.run_wi for g in got]), np.concatenate([g.run_off + sum(
                           x.ops.size for x in got[:k]) for k, g in enumerate(got)]).astype(np.uint64),
                       np.concatenate([g.run_len for g in got]), np.concatenate([g.ops for g in got]))
    # what rank `rank` holds equals shard `rank` of the whole trace routed in one process
    ref = S.route(whole, world)[rank]
    same = bool(np.array_equal(mine_all.mem, ref.mem) and np.array_equal(mine_all.br, ref.br) and
                np.array_equal(mine_all.run_wi, ref.run_wi) and np.array_equal(mine_all.run_len, ref.run_len))
    coc, ints, hist = _distributions(_trace_of(mine_all, tr.n_opcodes))
    # the exchange of the exported distributions: a sum over ranks
    flat_ints = torch.tensor(ints, dtype=torch.int64)
    dist.all_reduce(flat_ints)
    h = torch.from_numpy(hist.astype(np.int64))
    dist.all_reduce(h)
    cocs = [None] * world
    dist.all_gather_object(cocs, coc)
    blobs = S.gather_blobs(bytes([rank]) * (10 + 7 * rank))
    if rank == 0:
        summed = []
        for n in range(11):
            acc = {}
            for c in cocs:
                for k, v in c[n].items():
                    acc[k] = acc.get(k, 0) + v
            summed.append(acc)
        q.put((same, summed, flat_ints.tolist(), h.numpy(), blobs))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_route_exchange_and_add_to_the_whole_invocation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    same, summed, ints, hist, blobs = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert same
    tr = random_trace(11, n_mem=4000, n_br=3000, n_wi=6, n_runs=60, n_ops=5000, addr_pool=900, n_sites=7,
                      addr_span_bits=16)
    coc, whole_ints, whole_hist = _distributions(tr)
    for n in range(11):
        assert summed[n] == coc[n], n
    # totals, uniques, sites, patterns, barriers, ITB and IPT counts all add over whole units
    assert ints == whole_ints
    assert np.array_equal(hist.astype(np.uint64), whole_hist)
    assert blobs == [bytes([0]) * 10, bytes([1]) * 17]
