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


def _nbytes(t) -> int:
    return t.numel() * t.element_size() if hasattr(t, "element_size") else t.nbytes


def _records(t, size: int, what: str) -> int:
    """Number of `size`-byte records in a buffer; its bytes must be whole records."""
    nb = _nbytes(t)
    if nb % size:
        raise ValueError(f"{what}: {nb} bytes is not a whole number of {size}-byte records")
    return nb // size


def _elements(t, size: int, what: str) -> int:
    """Number of elements of a table whose elements must be `size` bytes wide."""
    es = t.element_size() if hasattr(t, "element_size") else t.itemsize
    if es != size:
        raise ValueError(f"{what} must have {size}-byte elements, not {es}")
    return t.numel() if hasattr(t, "numel") else t.size


class Characterizer:
    """One AIWC invocation at a time on one device (a handle of the C ABI)."""

    def __init__(self, device: int = 0, stream=None, history_len: int = 16, cover=(9, 10), n_opcodes: int = 65535,
                 space_mask: int = 0xF, precision: int = 0, plan: int = 0, max_work_items: int = 0,
                 hbm_budget: int = 0, table_slots: int = 0, partitions: int = 0, byte_addresses: int = 0,
                 history_scope: int = 0, defer_pushes: int = 0):
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
                                       byte_addresses=byte_addresses, history_scope=history_scope,
                                       defer_pushes=defer_pushes)
        self.h = aiwc_create(self.cfg)
        self._keep = []  # device inputs must outlive the next compute

    def push_mem(self, events) -> None:
        """events: (n, 2) int64 tensor / array holding 16-byte aiwc_mem_event records."""
        p, dev = _ptr(events)
        aiwc_push_mem(self.h, p, _records(events, 16, "memory events"), dev)
        if dev:
            self._keep.append(events)

    def push_branch(self, events) -> None:
        """events: (n,) int64 tensor / array holding 8-byte aiwc_branch_event records."""
        p, dev = _ptr(events)
        aiwc_push_branch(self.h, p, _records(events, 8, "branch events"), dev)
        if dev:
            self._keep.append(events)

    def push_instr(self, work_item: int, ops) -> None:
        """ops: (n,) int16 / uint16 opcodes of one work-item, 0xFFFF = barrier."""
        p, dev = _ptr(ops)
        aiwc_push_instr(self.h, work_item, p, _elements(ops, 2, "opcodes"), dev)
        if dev:
            self._keep.append(ops)

    def push_widths(self, widths) -> None:
        """widths: (n,) int16 / uint16 result widths of executed instructions."""
        p, dev = _ptr(widths)
        aiwc_push_widths(self.h, p, _elements(widths, 2, "widths"), dev)
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
        n_runs = _elements(run_wi, 4, "run_wi")
        if _elements(run_off, 8, "run_off") != n_runs or _elements(run_len, 8, "run_len") != n_runs:
            raise ValueError("run_wi, run_off and run_len must have one entry per run")
        n_ops = _elements(ops, 2, "opcodes")
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
