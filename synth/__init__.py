"""Seeded synthetic event traces for the AIWC metric reduction.

This module only *produces input event streams*; it holds none of the metric
arithmetic. Both the CPU oracle (``oracle/``) and the CUDA library consume
what it makes. Every value is a pure function of ``(seed, stream, index)``
through a counter-based hash (the SplitMix64 output function, Steele, Lea &
Flood 2014), written with wrapping int64 torch ops so the same call yields
bit-identical streams on the CPU and on a CUDA device.

Event layouts (little-endian, the byte layout the C ABI reads):

* memory event, 16 B: ``u64 addr | u32 work_item | u8 size | u8 flags | u16 0``
  with ``flags`` bit 0 = store, bits 1-2 = address space (0 global, 1 local,
  2 constant, 3 private). Held as an ``int64`` tensor of shape ``(n, 2)``.
* branch event, 8 B: ``u32 site | u32 (work_item | taken << 31)``. Held as an
  ``int64`` tensor of shape ``(n,)``.
* instruction stream: ``u16`` opcodes (``0xFFFF`` = barrier marker) held as
  ``int16``, plus a run table ``(work_item, offset, length)`` of per-work-item
  program-order runs.
"""
from .traces import (  # noqa: F401
    Trace, mix64, hash3, u01, pack_mem, pack_branch,
    tiny, large, large_mem, large_branch, large_instr, precision, batched, serving_jobs, pattern_trace,
    BARRIER_I16,
)
