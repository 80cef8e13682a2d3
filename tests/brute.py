"""Brute-force restatement of the AIWC metrics for tiny traces (pure Python).

Written independently of ``oracle/`` and in a different style: quadratic
scans over the raw event lists instead of sorts and maps, so that a mistake in
one is unlikely to be repeated in the other. Used only on traces of at most a
few hundred events.
"""
from __future__ import annotations

import math

import numpy as np

ADDR_LIMIT = 1 << 61


def decode(trace):
    """Return (mem, br, runs, ops) as plain Python lists."""
    mem = []
    if trace.mem is not None and trace.mem.shape[0]:
        raw = trace.mem.cpu().contiguous().numpy().view(np.uint8).reshape(-1, 16)
        for row in raw:
            addr = int.from_bytes(bytes(row[0:8]), "little")
            wi = int.from_bytes(bytes(row[8:12]), "little")
            flags = int(row[13])
            mem.append((addr, wi, flags & 1, (flags >> 1) & 3, int(row[12])))
    br = []
    if trace.br is not None and trace.br.shape[0]:
        raw = trace.br.cpu().contiguous().numpy().view(np.uint32).reshape(-1, 2)
        for site, wt in raw:
            br.append((int(site), int(wt) & 0x7FFFFFFF, int(wt) >> 31))
    ops = [] if trace.ops is None else [int(x) & 0xFFFF for x in trace.ops.cpu().tolist()]
    runs = []
    if trace.run_wi is not None:
        for w, o, n in zip(trace.run_wi.tolist(), trace.run_off.tolist(), trace.run_len.tolist()):
            runs.append((int(w) & 0xFFFFFFFF, int(o), int(n)))
    return mem, br, runs, ops


def _cover(counts, num, den):
    total = sum(counts)
    if total == 0:
        return 0
    # quadratic selection of the largest remaining count, one at a time
    left = list(counts)
    taken = 0
    k = 0
    while left:
        best = max(range(len(left)), key=lambda i: left[i])
        taken += left.pop(best)
        k += 1
        if den * taken >= num * total:
            return k
    return k


def _median(vals):
    if not vals:
        return 0, 0, 0.0
    # the i-th smallest value by counting, without sorting
    def kth(k):
        for v in vals:
            below = sum(1 for x in vals if x < v)
            equal = sum(1 for x in vals if x == v)
            if below <= k < below + equal:
                return v
        raise AssertionError
    m = len(vals)
    lo, hi = kth((m - 1) // 2), kth(m // 2)
    return lo, hi, (lo + hi) / 2.0


def metrics(trace, history_len=16, cover_num=9, cover_den=10, n_opcodes=None, space_mask=0xF,
            byte_addresses=0, history_scope=0):
    mem, br, runs, ops = decode(trace)
    nop = trace.n_opcodes if n_opcodes is None else n_opcodes
    out = {}
    wis = []

    # memory
    keys, rw = [], []
    for addr, wi, st, sp, size in mem:
        wis.append(wi)
        if addr >= ADDR_LIMIT:
            raise ValueError("address outside the 61-bit domain")
        touched = [addr + b for b in range(size)] if byte_addresses else [addr]
        if touched and touched[-1] >= ADDR_LIMIT:
            raise ValueError("a touched byte outside the 61-bit domain")
        if (space_mask >> sp) & 1:
            for a in touched:
                keys.append((sp, a))
                rw.append(st)
    N = len(keys)
    out["total_reads"] = sum(1 for s in rw if s == 0)
    out["total_writes"] = sum(1 for s in rw if s == 1)
    first = [i for i in range(N) if all(keys[j] != keys[i] for j in range(i))]
    out["footprint"] = len(first)
    out["unique_reads"] = sum(1 for i in range(N) if rw[i] == 0 and
                              all(not (keys[j] == keys[i] and rw[j] == 0) for j in range(i)))
    out["unique_writes"] = sum(1 for i in range(N) if rw[i] == 1 and
                               all(not (keys[j] == keys[i] and rw[j] == 1) for j in range(i)))
    counts0 = [sum(1 for k in keys if k == keys[i]) for i in first]
    out["footprint_cover"] = _cover(counts0, cover_num, cover_den)
    ent = []
    for n in range(11):
        g = [(sp, a >> n) for sp, a in keys]
        heads = [i for i in range(N) if all(g[j] != g[i] for j in range(i))]
        terms = []
        for i in heads:
            c = sum(1 for x in g if x == g[i])
            p = c / N
            terms.append(-p * math.log2(p))
        ent.append(math.fsum(terms) if N else 0.0)
    out["entropy"] = ent

    # branches: position of each event in its history -- the site's (work-item,
    # push order) sequence, or with history_scope=1 the (site, work-item)'s
    # push-order sequence
    B = len(br)
    for _, wi, _ in br:
        wis.append(wi)
    pos = []
    for e, (s, w, _) in enumerate(br):
        if history_scope:
            pos.append(sum(1 for f, (s2, w2, _) in enumerate(br) if s2 == s and w2 == w and f < e))
        else:
            pos.append(sum(1 for f, (s2, w2, _) in enumerate(br) if s2 == s and (w2 < w or (w2 == w and f < e))))
    sites = []
    for s, _, _ in br:
        if s not in sites:
            sites.append(s)
    out["branch_sites"] = len(sites)
    out["branch_cover"] = _cover([sum(1 for b in br if b[0] == s) for s in sites], cover_num, cover_den)
    out["branch_events"] = B

    def outcome(site, wi, p):
        for e, b in enumerate(br):
            if b[0] == site and (not history_scope or b[1] == wi) and pos[e] == p:
                return b[2]
        raise AssertionError

    h = history_len
    pats = []  # (site, history tuple, outcome)
    for e, (s, w, t) in enumerate(br):
        if pos[e] >= h:
            hist = tuple(outcome(s, w, pos[e] - h + k) for k in range(h))
            pats.append(((s, hist), t))
    seen = []
    minsum = 0
    for key, _ in pats:
        if key in seen:
            continue
        seen.append(key)
        n_ = sum(1 for k2, _ in pats if k2 == key)
        t_ = sum(t for k2, t in pats if k2 == key)
        minsum += min(t_, n_ - t_)
    out["branch_patterns"] = len(pats)
    out["branch_minsum"] = minsum
    out["albe"] = 2.0 * minsum / len(pats) if pats else 0.0
    # Yokota (reading): sum over sites of the site's share of predicted outcomes
    # times the entropy of its history distribution, in units of h bits
    terms = []
    for site in sorted({k[0] for k, _ in pats}):
        hs = [k[1] for k, _ in pats if k[0] == site]
        for hist in sorted(set(hs)):
            q = hs.count(hist) / len(hs)
            terms.append(len(hs) / len(pats) * -q * math.log2(q))
    out["yokota"] = max(0.0, math.fsum(terms) / h) if pats else 0.0

    # instructions: concatenate each work-item's runs, split at barriers
    order = []
    streams = {}
    for w, o, n in runs:
        if o > len(ops) or n > len(ops) - o:
            raise ValueError("run past the opcode array")
        wis.append(w)
        if w not in streams:
            streams[w] = []
            order.append(w)
        streams[w].extend(ops[o:o + n])
    hist = [0] * nop
    itb, ipt = [], []
    barriers = 0
    for w in order:
        seg = 0
        for op in streams[w]:
            if op == 0xFFFF:
                itb.append(seg)
                seg = 0
                barriers += 1
            else:
                if op >= nop:
                    raise ValueError("invalid opcode")
                hist[op] += 1
                seg += 1
        itb.append(seg)
        ipt.append(sum(1 for op in streams[w] if op != 0xFFFF))
    out["total_instructions"] = sum(hist)
    out["unique_opcodes"] = sum(1 for c in hist if c)
    out["opcode_cover"] = _cover([c for c in hist if c], cover_num, cover_den)
    out["barriers"] = barriers
    for name, vals in (("itb", itb), ("ipt", ipt)):
        lo, hi, med = _median(vals)
        out[f"{name}_count"] = len(vals)
        out[f"{name}_min"] = min(vals) if vals else 0
        out[f"{name}_max"] = max(vals) if vals else 0
        out[f"{name}_median_lo"], out[f"{name}_median_hi"], out[f"{name}_median"] = lo, hi, med
    out["opcode_hist"] = hist
    distinct_wi = []
    for w in wis:
        if w not in distinct_wi:
            distinct_wi.append(w)
    out["work_items"] = len(distinct_wi)
    return out
