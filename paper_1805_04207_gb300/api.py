"""Convenience wrapper: push torch tensors (CUDA or host) and compute.

Argument marshalling only -- every reduction step runs in libaiwc.so.
"""
from __future__ import annotations

import numpy as np

from . import (aiwc_compute, aiwc_compute_batch, aiwc_config_default, aiwc_create, aiwc_destroy, aiwc_device_bytes, aiwc_push_branch,
               aiwc_push_instr, aiwc_push_instr_runs, aiwc_push_widths, aiwc_push_mem, aiwc_set_stage_timing, aiwc_stage_times)


def _ptr(t):
    """(address, on_device) of a contiguous torch tensor or numpy array.

    The address is the caller's own buffer: anything that would need a
    temporary copy (a list, a strided view) is refused, since the copy would
    be freed before the library reads it."""
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return t.data_ptr(), bool(t.is_cuda)
    if not isinstance(t, np.ndarray) or not t.flags.c_contiguous:
        raise ValueError("host input must be a contiguous torch tensor or numpy array")
    return t.ctypes.data, False


class Characterizer:
    """One AIWC invocation at a time on one device (a handle of the C ABI)."""

    def __init__(self, device: int = 0, stream=None, history_len: int = 16, cover=(9, 10), n_opcodes: int = 65535,
                 space_mask: int = 0xF, precision: int = 0, plan: int = 0, max_work_items: int = 0,
                 hbm_budget: int = 0, table_slots: int = 0, partitions: int = 0, byte_addresses: int = 0,
                 history_scope: int = 0):
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream(device).cuda_stream
            except Exception:
                stream = 0
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self.n_opcodes = n_opcodes
        self.cfg = aiwc_config_default(device=device, cuda_stream=stream or None, history_len=history_len,
                                       cover_num=cover[0], cover_den=cover[1], n_opcodes=n_opcodes,
                                       space_mask=space_mask, precision=precision, plan=plan,
                                       max_work_items=max_work_items, hbm_budget=hbm_budget,
                                       table_slots=table_slots, partitions=partitions,
                                       byte_addresses=byte_addresses, history_scope=history_scope)
        self.h = aiwc_create(self.cfg)
        self._keep = []  # device inputs must outlive the next compute

    def push_mem(self, events) -> None:
        """events: (n, 2) int64 tensor / array holding 16-byte aiwc_mem_event records."""
        p, dev = _ptr(events)
        n = events.numel() // 2 if hasattr(events, "numel") else np.asarray(events).size // 2
        aiwc_push_mem(self.h, p, n, dev)
        if dev:
            self._keep.append(events)

    def push_branch(self, events) -> None:
        """events: (n,) int64 tensor / array holding 8-byte aiwc_branch_event records."""
        p, dev = _ptr(events)
        n = events.numel() if hasattr(events, "numel") else np.asarray(events).size
        aiwc_push_branch(self.h, p, n, dev)
        if dev:
            self._keep.append(events)

    def push_instr(self, work_item: int, ops) -> None:
        """ops: (n,) int16 / uint16 opcodes of one work-item, 0xFFFF = barrier."""
        p, dev = _ptr(ops)
        n = ops.numel() if hasattr(ops, "numel") else np.asarray(ops).size
        aiwc_push_instr(self.h, work_item, p, n, dev)
        if dev:
            self._keep.append(ops)

    def push_widths(self, widths) -> None:
        """widths: (n,) int16 / uint16 result widths of executed instructions."""
        p, dev = _ptr(widths)
        n = widths.numel() if hasattr(widths, "numel") else np.asarray(widths).size
        aiwc_push_widths(self.h, p, n, dev)
        if dev:
            self._keep.append(widths)

    def push_instr_runs(self, run_wi, run_off, run_len, ops) -> None:
        """run_wi: int32/uint32; run_off, run_len: int64; ops: int16/uint16; all on one side."""
        pw, d1 = _ptr(run_wi)
        po, d2 = _ptr(run_off)
        pl, d3 = _ptr(run_len)
        pp, d4 = _ptr(ops)
        if len({d1, d2, d3, d4}) != 1:
            raise ValueError("run table and opcodes must all be on the device or all on the host")
        n_runs = run_wi.numel() if hasattr(run_wi, "numel") else np.asarray(run_wi).size
        n_ops = ops.numel() if hasattr(ops, "numel") else np.asarray(ops).size
        aiwc_push_instr_runs(self.h, pw, po, pl, n_runs, pp, n_ops, d1)
        if d1:
            self._keep.extend([run_wi, run_off, run_len, ops])

    def compute(self, want_hist: bool = True) -> dict:
        hist = np.zeros(self.n_opcodes, dtype=np.uint64) if want_hist else None
        try:
            out = aiwc_compute(self.h, hist)
        finally:
            self._keep.clear()
        if want_hist:
            out["opcode_hist"] = hist
        return out

    def set_stage_timing(self, on: bool) -> None:
        aiwc_set_stage_timing(self.h, on)

    def stage_times(self) -> dict:
        return aiwc_stage_times(self.h)

    def device_bytes(self) -> int:
        return aiwc_device_bytes(self.h)

    def close(self) -> None:
        if self.h:
            aiwc_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def push_trace(c: Characterizer, trace) -> None:
    """Pushes every stream of a synth.Trace-like object (run table in bulk)."""
    if trace.mem is not None and trace.mem.shape[0]:
        c.push_mem(trace.mem)
    if trace.br is not None and trace.br.shape[0]:
        c.push_branch(trace.br)
    if trace.run_wi is not None and trace.run_wi.shape[0]:
        c.push_instr_runs(trace.run_wi.to(dtype=_i32(trace.run_wi)), trace.run_off, trace.run_len, trace.ops)
    widths = getattr(trace, "widths", None)
    if widths is not None and widths.shape[0]:
        c.push_widths(widths)


def _i32(t):
    import torch
    return torch.int32


def characterize(trace, device: int = 0, **cfg) -> dict:
    """Metrics of one invocation given as a synth.Trace (tensors on the GPU or host)."""
    cfg.setdefault("n_opcodes", trace.n_opcodes)
    with Characterizer(device=device, **cfg) as c:
        push_trace(c, trace)
        return c.compute()


def compute_batch(chars, want_hist: bool = True) -> list[dict]:
    """Computes several Characterizers' invocations together (one CUDA graph)."""
    hists = [np.zeros(c.n_opcodes, dtype=np.uint64) if want_hist else None for c in chars]
    try:
        outs = aiwc_compute_batch([c.h for c in chars], hists)
    finally:
        for c in chars:
            c._keep.clear()
    if want_hist:
        for o, hh in zip(outs, hists):
            o["opcode_hist"] = hh
    return outs
