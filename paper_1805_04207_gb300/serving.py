"""Thin wrapper over the serving entry points of the C ABI (marshalling only)."""
from __future__ import annotations

import numpy as np

from . import (aiwc_config_default, aiwc_job_finish, aiwc_job_open, aiwc_job_poll, aiwc_job_push_branch,
               aiwc_job_push_instr_runs, aiwc_job_push_mem, aiwc_job_push_widths, aiwc_job_wait,
               aiwc_server_config_default,
               aiwc_server_create, aiwc_server_destroy, aiwc_server_stats)
from .api import _elements, _ptr, _records


class Job:
    """One admitted characterization job; push chunks, finish, then poll or wait."""

    def __init__(self, server: "Server", handle: int, n_opcodes: int):
        self.server = server
        self.j = handle
        self.n_opcodes = n_opcodes
        self._keep = []  # device chunks must outlive the reduction

    def push_mem(self, events) -> None:
        p, dev = _ptr(events)
        aiwc_job_push_mem(self.j, p, _records(events, 16, "memory events"), dev)
        if dev:
            self._keep.append(events)

    def push_branch(self, events) -> None:
        p, dev = _ptr(events)
        aiwc_job_push_branch(self.j, p, _records(events, 8, "branch events"), dev)
        if dev:
            self._keep.append(events)

    def push_widths(self, widths) -> None:
        p, dev = _ptr(widths)
        aiwc_job_push_widths(self.j, p, _elements(widths, 2, "widths"), dev)
        if dev:
            self._keep.append(widths)

    def push_instr_runs(self, run_wi, run_off, run_len, ops) -> None:
        ptrs = [_ptr(t) for t in (run_wi, run_off, run_len, ops)]
        dev = ptrs[0][1]
        if any(d != dev for _, d in ptrs):
            raise ValueError("run table and opcodes must all be on the device or all on the host")
        n_runs = _elements(run_wi, 4, "run_wi")
        if _elements(run_off, 8, "run_off") != n_runs or _elements(run_len, 8, "run_len") != n_runs:
            raise ValueError("run_wi, run_off and run_len must have one entry per run")
        aiwc_job_push_instr_runs(self.j, ptrs[0][0], ptrs[1][0], ptrs[2][0], n_runs, ptrs[3][0],
                                 _elements(ops, 2, "opcodes"), dev)
        if dev:
            self._keep.extend([run_wi, run_off, run_len, ops])

    def finish(self) -> None:
        aiwc_job_finish(self.j)

    def poll(self, want_hist: bool = False):
        hist = np.zeros(self.n_opcodes, dtype=np.uint64) if want_hist else None
        out = aiwc_job_poll(self.j, hist)
        if out is not None:
            self._keep.clear()
            if want_hist:
                out["opcode_hist"] = hist
        return out

    def wait(self, want_hist: bool = False) -> dict:
        hist = np.zeros(self.n_opcodes, dtype=np.uint64) if want_hist else None
        out = aiwc_job_wait(self.j, hist)
        self._keep.clear()
        if want_hist:
            out["opcode_hist"] = hist
        return out


class Server:
    def __init__(self, device: int = 0, max_jobs: int = 32, workers: int = 4, hbm_budget: int = 120 << 30):
        self.cfg = aiwc_server_config_default(device=device, max_jobs=max_jobs, workers=workers,
                                              hbm_budget=hbm_budget)
        self.s = aiwc_server_create(self.cfg)

    def open(self, reserve_bytes: int, **cfg):
        """A Job, or None when the server has no slot or budget for it right now."""
        c = aiwc_config_default(**cfg)
        j = aiwc_job_open(self.s, c, reserve_bytes)
        return None if j is None else Job(self, j, c.n_opcodes)

    def stats(self) -> dict:
        return aiwc_server_stats(self.s)

    def close(self) -> None:
        if self.s:
            aiwc_server_destroy(self.s)
            self.s = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
