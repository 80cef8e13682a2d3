"""Small seeded random traces for the tests (numpy RNG; no metric arithmetic)."""
from __future__ import annotations

import numpy as np
import torch

from synth import Trace, pack_branch, pack_mem

BARRIER = -1


def random_trace(seed: int, n_mem: int = 40, n_br: int = 40, n_wi: int = 4, n_runs: int = 6,
                 n_ops: int = 60, addr_pool: int = 12, n_sites: int = 3, n_opcodes: int = 5,
                 spaces: int = 4, p_barrier: float = 0.15, addr_span_bits: int = 12,
                 size_choices=None) -> Trace:
    """A tiny trace over small alphabets so that collisions are frequent.

    Accesses are 4 bytes wide unless `size_choices` is given; their sizes are
    then drawn from it after every other draw (the rest of the trace is the
    same as without it).
    """
    rng = np.random.default_rng(seed)
    pool = rng.integers(0, 1 << addr_span_bits, size=addr_pool, dtype=np.int64)
    addr = pool[rng.integers(0, addr_pool, size=n_mem)]
    mem = pack_mem(torch.from_numpy(addr), torch.from_numpy(rng.integers(0, n_wi, n_mem)),
                   torch.full((n_mem,), 4, dtype=torch.int64),
                   torch.from_numpy(rng.integers(0, 2, n_mem)),
                   torch.from_numpy(rng.integers(0, spaces, n_mem)))
    br = pack_branch(torch.from_numpy(rng.integers(0, n_sites, n_br)),
                     torch.from_numpy(rng.integers(0, n_wi, n_br)),
                     torch.from_numpy(rng.integers(0, 2, n_br)))
    ops = rng.integers(0, n_opcodes, size=n_ops)
    ops[rng.random(n_ops) < p_barrier] = BARRIER
    cuts = np.sort(rng.choice(np.arange(1, n_ops), size=n_runs - 1, replace=False)) if n_runs > 1 else []
    bounds = [0, *cuts, n_ops]
    run_off = np.array(bounds[:-1], dtype=np.int64)
    run_len = np.diff(np.array(bounds, dtype=np.int64))
    run_wi = rng.integers(0, n_wi, size=n_runs)
    if size_choices is not None:
        sizes = np.asarray(size_choices, dtype=np.int64)[rng.integers(0, len(size_choices), n_mem)]
        raw = mem.view(torch.uint8).reshape(-1, 16).clone()
        raw[:, 12] = torch.from_numpy(sizes.astype(np.uint8))
        mem = raw.view(torch.int64).reshape(-1, 2)
    return Trace(f"rand{seed}", mem, br, torch.from_numpy(ops.astype(np.int16)),
                 torch.from_numpy(run_wi.astype(np.int64)), torch.from_numpy(run_off),
                 torch.from_numpy(run_len), n_opcodes=n_opcodes)


def mem_only(addrs, stores=None, spaces=None, wis=None, sizes=None) -> Trace:
    n = len(addrs)
    sz = torch.full((n,), 4, dtype=torch.int64) if sizes is None else torch.tensor(sizes, dtype=torch.int64)
    a = torch.tensor(addrs, dtype=torch.int64)
    st = torch.zeros(n, dtype=torch.int64) if stores is None else torch.tensor(stores, dtype=torch.int64)
    sp = torch.zeros(n, dtype=torch.int64) if spaces is None else torch.tensor(spaces, dtype=torch.int64)
    wi = torch.zeros(n, dtype=torch.int64) if wis is None else torch.tensor(wis, dtype=torch.int64)
    return Trace("mem", pack_mem(a, wi, sz, st, sp))


def branch_only(sites, wis, taken) -> Trace:
    return Trace("br", br=pack_branch(torch.tensor(sites, dtype=torch.int64),
                                      torch.tensor(wis, dtype=torch.int64),
                                      torch.tensor(taken, dtype=torch.int64)))


def instr_only(runs, n_opcodes=8) -> Trace:
    """runs: list of (work_item, [ops...]) in push order; -1 is a barrier."""
    ops, wi, off, ln = [], [], [], []
    for w, seq in runs:
        wi.append(w)
        off.append(len(ops))
        ln.append(len(seq))
        ops.extend(seq)
    return Trace("ins", ops=torch.tensor(ops, dtype=torch.int16), run_wi=torch.tensor(wi, dtype=torch.int64),
                 run_off=torch.tensor(off, dtype=torch.int64), run_len=torch.tensor(ln, dtype=torch.int64),
                 n_opcodes=n_opcodes)
