"""Sharded invocations: one kernel invocation reduced by several ranks.

Each rank holds a slice of the invocation's streams (host arrays, in push
order: rank r's slice comes before rank r+1's). libaiwc.so routes the slice
into one shard per rank, keeping every unit of the method whole (memory
superblocks, branch sites, work-items' runs); an all-to-all hands shard s of
every rank to rank s; each rank pushes what it received in source-rank order
and exports its exact distributions (aiwc_shard_export); the blobs are
gathered and libaiwc.so adds them and finalises once (aiwc_shard_merge), so
every rank obtains the metrics of the whole invocation, identical to a
single-device reduction. Sec. V of the paper adds each work-group's results
into the kernel's global state; this is the same addition across ranks.

This module only marshals arguments and moves bytes with torch.distributed
(gloo for host buffers; the same calls carry CUDA tensors over NCCL).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import (aiwc_shard_export, aiwc_shard_merge, aiwc_shard_route_branch, aiwc_shard_route_mem,
               aiwc_shard_route_runs)


def _u8(a, width: int) -> np.ndarray:
    if a is None:
        return np.zeros(0, dtype=np.uint8)
    if hasattr(a, "detach"):
        a = a.detach().cpu().contiguous().numpy()
    b = np.ascontiguousarray(a).view(np.uint8).reshape(-1)
    if b.size % width:
        raise ValueError(f"buffer of {b.size} bytes is not a whole number of {width}-byte records")
    return b


def _arr(a, dtype) -> np.ndarray:
    if a is None:
        return np.zeros(0, dtype=dtype)
    if hasattr(a, "detach"):
        a = a.detach().cpu().contiguous().numpy()
    return np.ascontiguousarray(a).astype(dtype, copy=False)


@dataclass
class Slice:
    """Host streams of (part of) one invocation, as raw records."""
    mem: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint8))      # 16-byte memory events
    br: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint8))       # 8-byte branch events
    run_wi: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint32))
    run_off: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint64))
    run_len: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint64))
    ops: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint16))
    widths: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint16))

    @classmethod
    def of_trace(cls, trace) -> "Slice":
        """A synth.Trace-like object (torch tensors or numpy arrays) as a host slice."""
        return cls(_u8(trace.mem, 16), _u8(trace.br, 8), _arr(trace.run_wi, np.uint32),
                   _arr(trace.run_off, np.uint64), _arr(trace.run_len, np.uint64),
                   _u8(trace.ops, 2).view(np.uint16), _u8(getattr(trace, "widths", None), 2).view(np.uint16))

    def pack(self) -> np.ndarray:
        """One byte array: six lengths, then the six streams (widths stay with their rank)."""
        parts = [self.mem, self.br, self.run_wi, self.run_off, self.run_len, self.ops]
        raw = [np.ascontiguousarray(p).view(np.uint8).reshape(-1) for p in parts]
        head = np.array([r.size for r in raw], dtype=np.uint64).view(np.uint8)
        return np.concatenate([head, *raw])

    @classmethod
    def unpack(cls, b: np.ndarray) -> "Slice":
        n = np.frombuffer(b[:48].tobytes(), dtype=np.uint64)
        at = 48
        out = []
        for k, dt in zip(range(6), (np.uint8, np.uint8, np.uint32, np.uint64, np.uint64, np.uint16)):
            out.append(np.frombuffer(b[at:at + int(n[k])].tobytes(), dtype=dt).copy())
            at += int(n[k])
        return cls(*out)


def route(sl: Slice, n_shards: int, byte_addresses: int = 0) -> list[Slice]:
    """Shard s of a rank's slice for every s (libaiwc.so's routing)."""
    mem, mc = aiwc_shard_route_mem(n_shards, sl.mem, byte_addresses)
    br, bc = aiwc_shard_route_branch(n_shards, sl.br)
    wi, off, ln, ops, rc, oc = aiwc_shard_route_runs(n_shards, sl.run_wi, sl.run_off, sl.run_len, sl.ops)
    out = []
    m0 = b0 = r0 = o0 = 0
    for s in range(n_shards):
        m1, b1, r1, o1 = m0 + int(mc[s]), b0 + int(bc[s]), r0 + int(rc[s]), o0 + int(oc[s])
        out.append(Slice(mem[16 * m0:16 * m1], br[8 * b0:8 * b1], wi[r0:r1], off[r0:r1], ln[r0:r1], ops[o0:o1]))
        m0, b0, r0, o0 = m1, b1, r1, o1
    return out


def _dist():
    import torch.distributed as dist
    return dist


def exchange(shards: list[Slice], group=None) -> list[Slice]:
    """All-to-all: sends shards[s] to rank s; returns what every rank sent
    here, in source-rank order."""
    import torch
    dist = _dist()
    world = dist.get_world_size(group)
    if len(shards) != world:
        raise ValueError("one shard per rank")
    packed = [s.pack() for s in shards]
    send_sizes = torch.tensor([p.size for p in packed], dtype=torch.int64)
    recv_sizes = torch.empty(world, dtype=torch.int64)
    dist.all_to_all_single(recv_sizes, send_sizes, group=group)
    send = torch.from_numpy(np.concatenate(packed))
    recv = torch.empty(int(recv_sizes.sum()), dtype=torch.uint8)
    dist.all_to_all_single(recv, send, output_split_sizes=recv_sizes.tolist(),
                           input_split_sizes=send_sizes.tolist(), group=group)
    r = recv.numpy()
    out, at = [], 0
    for k in recv_sizes.tolist():
        out.append(Slice.unpack(r[at:at + k]))
        at += k
    return out


def gather_blobs(blob: bytes, group=None) -> list[bytes]:
    """Every rank's blob, in rank order, on every rank."""
    import torch
    dist = _dist()
    world = dist.get_world_size(group)
    size = torch.tensor([len(blob)], dtype=torch.int64)
    sizes = [torch.empty(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, size, group=group)
    cap = max(int(s.item()) for s in sizes)
    mine = torch.zeros(cap, dtype=torch.uint8)
    mine[:len(blob)] = torch.frombuffer(bytearray(blob), dtype=torch.uint8)
    bufs = [torch.empty(cap, dtype=torch.uint8) for _ in range(world)]
    dist.all_gather(bufs, mine, group=group)
    return [bytes(b[:int(s.item())].numpy()) for b, s in zip(bufs, sizes)]


def push_slice(c, sl: Slice) -> None:
    """Pushes a host slice into a Characterizer (host buffers: copied before return)."""
    if sl.mem.size:
        c.push_mem(sl.mem)
    if sl.br.size:
        c.push_branch(sl.br)
    if sl.run_wi.size:
        c.push_instr_runs(sl.run_wi, sl.run_off, sl.run_len, sl.ops if sl.ops.size else np.zeros(1, np.uint16))
    if sl.widths.size:
        c.push_widths(sl.widths)


def reduce_sharded(c, mine: Slice, group=None, want_hist: bool = True) -> dict:
    """Metrics of the whole invocation whose slices the ranks of `group` hold.

    `c` is this rank's Characterizer (the same metric configuration on every
    rank); every rank returns the same result."""
    dist = _dist()
    world = dist.get_world_size(group)
    shards = route(mine, world, int(c.cfg.byte_addresses))
    for sl in exchange(shards, group):
        push_slice(c, sl)
    if mine.widths.size:  # SIMD statistics add over any split: widths stay with their rank
        c.push_widths(mine.widths)
    blobs = gather_blobs(aiwc_shard_export(c.h), group)
    hist = np.zeros(c.n_opcodes, dtype=np.uint64) if want_hist else None
    out = aiwc_shard_merge(c.h, blobs, hist)
    if want_hist:
        out["opcode_hist"] = hist
    return out
