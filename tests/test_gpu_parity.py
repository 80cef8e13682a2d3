"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integers, medians and the opcode histogram must match bit-exactly; every
entropy must be within 1e-9 bits (the FP64 tolerance), the linear branch
entropy within 1e-12 (it is one division of exact integers).
"""
from __future__ import annotations

import math

import numpy as np
import pytest
import torch

import oracle
import synth
from tests.helpers import branch_only, instr_only, mem_only, random_trace

pytestmark = pytest.mark.gpu

INT_FIELDS = ["total_instructions", "unique_opcodes", "opcode_cover", "work_items", "barriers",
              "itb_count", "itb_min", "itb_max", "itb_median_lo", "itb_median_hi",
              "ipt_count", "ipt_min", "ipt_max", "ipt_median_lo", "ipt_median_hi",
              "total_reads", "total_writes", "footprint", "footprint_cover", "unique_reads", "unique_writes",
              "branch_events", "branch_sites", "branch_cover", "branch_patterns", "branch_minsum",
              "simd_count", "simd_max", "simd_sum", "simd_sumsq"]
ENTROPY_TOL = 1e-9
# SIMD mean / SD and the Kiviat quantities are single FP64 divisions (and a
# square root) of exact integers: they agree to a few ulps
REAL_FIELDS = ["simd_mean", "simd_sd", "granularity", "barriers_per_instruction", "instructions_per_operand",
               "load_imbalance"]
REAL_RTOL = 1e-13


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_04207_gb300 as P
    return P


def assert_parity(g, o, entropy_tol=ENTROPY_TOL, hist=True):
    bad = [(f, g[f], o[f]) for f in INT_FIELDS if g[f] != o[f]]
    assert not bad, bad
    assert g["itb_median"] == o["itb_median"] and g["ipt_median"] == o["ipt_median"]
    for n in range(11):
        assert abs(g["entropy"][n] - o["entropy"][n]) <= entropy_tol, (n, g["entropy"][n], o["entropy"][n])
    assert abs(g["albe"] - o["albe"]) <= 1e-12  # FP64 in both precision modes
    assert abs(g["yokota"] - o["yokota"]) <= max(1e-12, entropy_tol)
    for r in ("unique_rw_ratio", "reread_ratio", "rewrite_ratio"):
        a, b = g[r], o[r]
        assert (math.isnan(a) and math.isnan(b)) or a == b, (r, a, b)
    for r in REAL_FIELDS:
        a, b = g[r], o[r]
        assert (math.isnan(a) and math.isnan(b)) or a == b or abs(a - b) <= REAL_RTOL * abs(b), (r, a, b)
    if hist:
        assert np.array_equal(np.asarray(g["opcode_hist"], dtype=np.uint64),
                              np.asarray(o["opcode_hist"], dtype=np.uint64))


def run_gpu(P, trace, on_device=True, split=1, single_runs=False, **cfg):
    cfg.setdefault("n_opcodes", trace.n_opcodes)
    tr = trace.to("cuda") if on_device else trace
    with P.Characterizer(**cfg) as c:
        for part in range(split):
            if tr.mem is not None and tr.mem.shape[0]:
                n = tr.mem.shape[0]
                c.push_mem(tr.mem[part * n // split:(part + 1) * n // split].contiguous())
            if tr.br is not None and tr.br.shape[0]:
                n = tr.br.shape[0]
                c.push_branch(tr.br[part * n // split:(part + 1) * n // split].contiguous())
        if tr.widths is not None and tr.widths.shape[0]:
            c.push_widths(tr.widths)
        if tr.run_wi is not None and tr.run_wi.shape[0]:
            if single_runs:
                for w, o, ln in zip(trace.run_wi.tolist(), trace.run_off.tolist(), trace.run_len.tolist()):
                    c.push_instr(int(w), tr.ops[o:o + ln].contiguous())
            else:
                R = tr.run_wi.shape[0]
                for part in range(split):
                    sl = slice(part * R // split, (part + 1) * R // split)
                    c.push_instr_runs(tr.run_wi[sl].to(torch.int32).contiguous(), tr.run_off[sl].contiguous(),
                                      tr.run_len[sl].contiguous(), tr.ops)
        return c.compute()


def test_tiny_workload(P):
    tr = synth.tiny()
    o = oracle.compute(tr)
    assert_parity(run_gpu(P, tr), o)
    assert_parity(run_gpu(P, tr, on_device=False), o)
    assert_parity(run_gpu(P, tr, single_runs=True), o)
    assert_parity(run_gpu(P, tr, on_device=False, single_runs=True, split=3), o)


@pytest.mark.parametrize("seed", range(40))
def test_random_tiny_traces(P, seed):  # noqa: D103 (plans alternate with the seed)
    rng = np.random.default_rng(20_000 + seed)
    tr = random_trace(seed, n_mem=int(rng.integers(0, 300)), n_br=int(rng.integers(0, 300)),
                      n_wi=int(rng.integers(1, 9)), n_runs=int(rng.integers(1, 12)),
                      n_ops=int(rng.integers(12, 400)), addr_pool=int(rng.integers(1, 64)),
                      n_sites=int(rng.integers(1, 5)), n_opcodes=int(rng.integers(1, 9)),
                      addr_span_bits=int(rng.integers(1, 40)))
    h = int(rng.choice([1, 2, 5, 16, 31]))
    mask = int(rng.choice([0xF, 0x1, 0x6]))
    o = oracle.compute(tr, history_len=h, space_mask=mask)
    g = run_gpu(P, tr, on_device=bool(seed % 2), split=1 + seed % 3, single_runs=seed % 4 == 3, history_len=h,
                space_mask=mask, plan=(seed // 2) % 2)
    assert_parity(g, o)


@pytest.mark.parametrize("plan", [0, 1])
@pytest.mark.parametrize("n_mem,n_br,n_wi,per_wi", [
    (300_000 + 12345, 200_001, 257, 1000),
    (4096 * 7, 4096 * 3, 64, 4096),
    (1_000_003, 1_000_003, 1000, 1001),
])
def test_large_shape_ragged(P, n_mem, n_br, n_wi, per_wi, plan):
    tr = synth.large(seed=3, n_mem=n_mem, n_br=n_br, n_wi=n_wi, per_wi=per_wi, zipf_distinct=1 << 16)
    o = oracle.compute(tr)
    assert_parity(run_gpu(P, tr, plan=plan), o)


def test_hash_plan_table_overflow_falls_back_to_sort(P):
    """A table far too small for the superblocks overflows; that invocation is
    finished by the sort plan, the next one gets a larger table -- results
    are identical either way."""
    tr = synth.large(seed=4, n_mem=400_000, n_br=1000, n_wi=4, per_wi=100, zipf_distinct=1 << 18)
    o = oracle.compute(tr)
    from paper_1805_04207_gb300.api import push_trace
    with P.Characterizer(n_opcodes=tr.n_opcodes, table_slots=64) as c:
        for _ in range(6):  # 64 -> 256 -> 1024 -> ... slots
            push_trace(c, tr.to("cuda"))
            assert_parity(c.compute(), o)


def test_empty_and_single_stream(P):
    for tr in (synth.Trace("empty"), mem_only([5]), branch_only([1], [2], [1]), instr_only([(3, [])]),
               instr_only([(3, [-1, -1])]), mem_only([0, 0, 0], stores=[1, 1, 1])):
        assert_parity(run_gpu(P, tr), oracle.compute(tr), hist=tr.ops is not None)


@pytest.mark.parametrize("plan", [0, 1])
def test_one_address_many_tiles(P, plan):
    # one run of equal keys spanning many tiles exercises the cross-tile fix-up
    tr = mem_only([1 << 20] * 200_000, stores=[i % 3 == 0 for i in range(200_000)])
    assert_parity(run_gpu(P, tr, plan=plan), oracle.compute(tr))
    tr = branch_only([9] * 100_000, list(range(100_000)), [int(i % 7 != 0) for i in range(100_000)])
    assert_parity(run_gpu(P, tr), oracle.compute(tr))


@pytest.mark.parametrize("plan", [0, 1])
def test_key_extremes_and_spaces(P, plan):
    top = (1 << 61) - 1
    addrs = [0, 1, top, top - 1, 1 << 60, 0, top] * 1000
    spaces = [0, 3, 3, 0, 1, 2, 2] * 1000
    tr = mem_only(addrs, stores=[i % 2 for i in range(len(addrs))], spaces=spaces)
    for mask in (0xF, 0x9, 0x2):
        assert_parity(run_gpu(P, tr, space_mask=mask, plan=plan), oracle.compute(tr, space_mask=mask))


@pytest.mark.parametrize("plan", [0, 1])
def test_all_distinct_addresses(P, plan):
    n = 150_000
    tr = mem_only(list(range(0, 8 * n, 8)))
    assert_parity(run_gpu(P, tr, plan=plan), oracle.compute(tr))


@pytest.mark.parametrize("shift", [0, 1, 2, 3, 4])
def test_address_alignment_shifts(P, shift):
    """Every address a multiple of 2^shift: the hash plan walks superblocks in
    compressed form and copies the lowest skip levels; segments span few
    events, a few hundred, and (one hot superblock) more than 2^14."""
    rng = np.random.default_rng(100 + shift)
    n_wide, n_hot = 250_000, 40_000
    idx = np.concatenate([rng.integers(0, 1 << 17, n_wide),                      # spread over many superblocks
                          (1 << 20) + rng.integers(0, 2048 >> min(shift, 3), n_hot),  # one hot superblock
                          rng.zipf(1.3, 30_000) % (1 << 12)])                      # heavy repeats
    addr = (idx.astype(np.int64) << shift) + (5 << 33)
    n = addr.shape[0]
    perm = rng.permutation(n)
    tr = mem_only(addr[perm].tolist(), stores=(rng.random(n) < 0.3).astype(np.int64).tolist(),
                  spaces=rng.integers(0, 2, n).tolist())
    assert_parity(run_gpu(P, tr, plan=0, table_slots=1 << 16), oracle.compute(tr))


def _site_trace(seed, n, n_sites, wi_sorted=True):
    rng = np.random.default_rng(seed)
    sites = rng.integers(0, n_sites, n)
    wis = np.arange(n) // 64 if wi_sorted else rng.integers(0, 1 << 16, n)
    p_site = rng.random(n_sites)
    taken = (rng.random(n) < p_site[sites]).astype(np.int64)
    return branch_only(sites.tolist(), wis.tolist(), taken.tolist())


@pytest.mark.parametrize("n,n_sites,wi_sorted,split,h", [
    ((1 << 16) + 3, 4096, True, 1, 16),       # one ragged tile past four
    (1_100_000 + 77, 4000, True, 3, 16),      # three pushes
    (2_200_003, 3000, True, 2, 16),           # more than one scan chunk of 64 tiles
    (300_001, 50, True, 2, 3),                # few, long sites
    (200_000, 5000, True, 1, 16),             # site ids >= 4096: radix sort
    (200_000, 1000, False, 1, 16),            # work-items out of order: radix sort
])
def test_site_counting_sort(P, n, n_sites, wi_sorted, split, h):
    """The stable counting sort by site (work-items in order, site ids below
    4096) and its fallbacks give the oracle's branch metrics."""
    tr = _site_trace(7 + n_sites, n, n_sites, wi_sorted)
    assert_parity(run_gpu(P, tr, split=split, history_len=h), oracle.compute(tr, history_len=h))


def _long_site_trace(seed, n, weights, wi_sorted=True):
    """Branch events over len(weights) sites drawn with those weights: site 0
    is always taken (one history pattern predicts nearly all its outcomes),
    the others are taken with a probability of their own."""
    rng = np.random.default_rng(seed)
    w = np.asarray(weights, dtype=float)
    sites = rng.choice(len(w), n, p=w / w.sum())
    wis = np.arange(n) // 64 if wi_sorted else rng.integers(0, 1 << 16, n)
    p_site = rng.random(len(w))
    p_site[0] = 1.0
    taken = (rng.random(n) < p_site[sites]).astype(np.int64)
    return branch_only(sites.tolist(), wis.tolist(), taken.tolist())


@pytest.mark.parametrize("n,weights,wi_sorted,h,scope", [
    (400_003, [1, 1, 1], True, 16, 0),                # counting sort; about 133K outcomes per site
    (400_003, [1, 1, 1], False, 16, 0),               # work-items out of order: radix sort
    (300_001, [6, 1] + [0.01] * 300, True, 17, 0),    # long sites among short ones, two passes of bins
    (250_007, [3, 1], False, 5, 1),                   # one history per (site, work-item)
    (200_003, [5, 1, 1], True, 1, 1),
])
def test_long_sites(P, n, weights, wi_sorted, h, scope):
    """Sites longer than 65,535 outcomes are counted in chunks on the per-site
    path; the branch metrics equal the oracle's and the global path's."""
    tr = _long_site_trace(900 + n % 97, n, weights, wi_sorted)
    o = oracle.compute(tr, history_len=h, history_scope=scope)
    for split, plan in ((1, 0), (3, 0), (1, 1)):
        assert_parity(run_gpu(P, tr, split=split, history_len=h, history_scope=scope, plan=plan), o)


@pytest.mark.parametrize("h,scope", [(1, 0), (16, 0), (3, 1)])
def test_site_lengths_at_the_chunk_limits(P, h, scope):
    """Sites of 65,536 and 65,535 outcomes (one above and at the per-block
    limit), one of exactly two chunks plus h + 1, interleaved in push order."""
    rng = np.random.default_rng(h + 10 * scope)
    sites = np.concatenate([np.zeros(65_536, np.int64), np.ones(65_535, np.int64),
                            np.full(2 * 16_384 + h + 1, 2, np.int64), np.full(5, 3, np.int64)])
    sites = sites[rng.permutation(sites.size)]
    n = sites.size
    wis = np.arange(n) // 100
    taken = (rng.random(n) < np.array([0.9, 0.5, 0.2, 0.5])[sites]).astype(np.int64)
    tr = branch_only(sites.tolist(), wis.tolist(), taken.tolist())
    o = oracle.compute(tr, history_len=h, history_scope=scope)
    for split, plan in ((1, 0), (2, 0), (1, 1)):
        assert_parity(run_gpu(P, tr, split=split, history_len=h, history_scope=scope, plan=plan), o)


def test_long_sites_in_a_batch(P):
    """Long sites in one batched graph, twice: with the counting sort (the
    per-site path certain on the host), and with more than 2^20 events
    arriving out of work-item order (the path chosen on the device)."""
    from paper_1805_04207_gb300.api import compute_batch, push_trace
    traces = [_long_site_trace(41, 400_003, [1, 1, 1], True), _long_site_trace(42, 1_200_001, [4, 2, 1, 1, 1], False),
              _site_trace(43, 70_000, 300, True), synth.tiny()]
    expect = [oracle.compute(t) for t in traces]
    chars = [P.Characterizer(n_opcodes=t.n_opcodes) for t in traces]
    try:
        for _ in range(2):
            for c, t in zip(chars, traces):
                push_trace(c, t.to("cuda"))
            for g, o in zip(compute_batch(chars), expect):
                assert_parity(g, o)
    finally:
        for c in chars:
            c.close()


def test_gated_branch_path_in_a_batch(P):
    """History length 17 with more than 65,535 branch events: the per-site
    path is not certain on the host, so the batched graph holds both branch
    paths (and the one-sweep pattern sort) behind the device's choice; twice,
    against the oracle."""
    from paper_1805_04207_gb300.api import compute_batch, push_trace
    traces = [_long_site_trace(51, 300_001, [6, 1] + [0.01] * 300, True), _site_trace(52, 90_000, 5000, False),
              synth.tiny()]
    expect = [oracle.compute(t, history_len=17) for t in traces]
    chars = [P.Characterizer(n_opcodes=t.n_opcodes, history_len=17) for t in traces]
    try:
        for _ in range(2):
            for c, t in zip(chars, traces):
                push_trace(c, t.to("cuda"))
            for g, o in zip(compute_batch(chars), expect):
                assert_parity(g, o)
    finally:
        for c in chars:
            c.close()


@pytest.mark.parametrize("n,offset,on_device", [(0, 0, True), (1, 0, True), (4099, 1, True), (300_001, 0, False),
                                                  (1_000_003, 3, True)])
def test_simd_widths(P, n, offset, on_device):
    """SIMD widths (Table I) pushed from host or device memory, aligned or
    not, in one or two pushes; every other metric is unaffected."""
    rng = np.random.default_rng(n + offset)
    w = rng.integers(0, 65536, n + offset, dtype=np.int64).astype(np.uint16).view(np.int16)
    widths = torch.from_numpy(w.copy())
    tr = instr_only([(0, [1, 2, -1, 3])], n_opcodes=8)
    with P.Characterizer(n_opcodes=8) as c:
        c.push_instr_runs(tr.run_wi.to(torch.int32), tr.run_off, tr.run_len, tr.ops)
        src = widths.cuda() if on_device else widths
        half = (n + offset) // 2
        if offset:
            c.push_widths(src[offset:half].contiguous() if not on_device else src[offset:half])
            c.push_widths(src[half:])
        else:
            c.push_widths(src)
        g = c.compute(want_hist=True)
    tr.widths = widths[offset:]
    assert_parity(g, oracle.compute(tr))


def test_aggregate_matches_oracle(P):
    """Sum and median over invocations (Sec. VI) of real GPU results."""
    runs = [run_gpu(P, synth.pattern_trace(k, c, f, seed=3, stream=i)) for i, (k, c, f) in
            enumerate([("zipf", 50_000, 9_000), ("stencil", 70_001, 20_000), ("gemm", 64_000, 16_384),
                       ("uniform", 20_000, 20_000)])]
    for mode, pm in (("sum", P.AGG_SUM), ("median", P.AGG_MEDIAN)):
        g = P.aiwc_aggregate(runs, pm)
        o = oracle.aggregate(runs, mode)
        for k, v in o.items():
            if k == "entropy":
                assert all(abs(a - b) <= 1e-12 * max(1.0, abs(b)) for a, b in zip(g[k], v)), k
            elif isinstance(v, float):
                assert (math.isnan(v) and math.isnan(g[k])) or g[k] == v or abs(g[k] - v) <= 1e-12 * abs(v), k
            else:
                assert g[k] == v, (k, g[k], v)


def test_value_overflow_paths(P):
    # ITB/IPT values above the shared (2048) and dense (65536) bins, opcode
    # counts above 1024, and work-items with many runs.
    runs = [(0, [1] * 70_000), (1, [2] * 3000 + [-1] + [3] * 100), (0, [4] * 10 + [-1]), (2, [])]
    runs += [(5, [k % 6] * 3 + [-1]) for k in range(500)]
    tr = instr_only(runs, n_opcodes=7)
    assert_parity(run_gpu(P, tr), oracle.compute(tr))
    assert_parity(run_gpu(P, tr, single_runs=True, on_device=False), oracle.compute(tr))


@pytest.mark.parametrize("h", [1, 2, 7, 16, 31])
def test_history_lengths(P, h):
    tr = synth.large(seed=5, n_mem=1000, n_br=300_000, n_wi=2, per_wi=100, zipf_distinct=1 << 10)
    assert_parity(run_gpu(P, tr, history_len=h), oracle.compute(tr, history_len=h))


def test_cover_fractions(P):
    tr = synth.large(seed=6, n_mem=200_000, n_br=50_000, n_wi=50, per_wi=500, zipf_distinct=1 << 12)
    for num, den in ((1, 2), (1, 1), (99, 100), (1, 1000)):
        assert_parity(run_gpu(P, tr, cover=(num, den)), oracle.compute(tr, cover_num=num, cover_den=den))


def test_handle_reuse_resets_state(P):
    a = synth.large(seed=7, n_mem=100_000, n_br=40_000, n_wi=30, per_wi=700, zipf_distinct=1 << 12)
    b = synth.tiny()
    with P.Characterizer(n_opcodes=256) as c:
        from paper_1805_04207_gb300.api import push_trace
        outs = []
        for tr in (a, b, a):
            push_trace(c, tr.to("cuda"))
            outs.append(c.compute())
    assert_parity(outs[0], oracle.compute(a, n_opcodes=256))
    assert_parity(outs[1], oracle.compute(b, n_opcodes=256))
    assert_parity(outs[2], outs[0])


def test_invalid_events_reported_then_handle_recovers(P):
    with P.Characterizer(n_opcodes=8) as c:
        c.push_mem(mem_only([1 << 61]).mem.cuda())
        with pytest.raises(P.AiwcError) as e:
            c.compute()
        assert e.value.status == P.AIWC_EINVAL
        tr = instr_only([(0, [9])], n_opcodes=8)
        c.push_instr(0, tr.ops.cuda())
        with pytest.raises(P.AiwcError) as e:
            c.compute()
        assert e.value.status == P.AIWC_EINVAL
        good = synth.tiny()
        from paper_1805_04207_gb300.api import push_trace
        c2 = P.Characterizer(n_opcodes=64)
        push_trace(c2, good.to("cuda"))
        assert_parity(c2.compute(), oracle.compute(good))
        c2.close()
        c.push_mem(mem_only([4, 4, 8]).mem.cuda())
        g = c.compute()
        assert (g["footprint"], g["total_reads"]) == (2, 3)
    with P.Characterizer(max_work_items=16) as c:
        c.push_branch(branch_only([1], [20], [1]).br.cuda())
        with pytest.raises(P.AiwcError):
            c.compute()


@pytest.mark.slow
def test_full_size_large_invocation(P):
    """The 2^28 / 2^26 / 2^30-event invocation in bench.py's launch configuration,
    against the oracle run on the host over the same inputs."""
    tr_dev = synth.large(device="cuda")
    g = run_gpu(P, tr_dev.to("cuda"))
    tr = tr_dev.to("cpu")
    del tr_dev
    torch.cuda.empty_cache()
    o = oracle.compute(tr)
    assert_parity(g, o)


@pytest.mark.parametrize("h", [3, 16])
def test_branch_order_detection_across_pushes(P, h):
    """Work-items in order inside each push but not across pushes must still
    give (work-item, program order) histories; in order everywhere takes the
    site-only sort."""
    rng = np.random.default_rng(99)
    n = 30_000
    sites = rng.integers(0, 7, n)
    taken = rng.integers(0, 2, n)
    wis = np.sort(rng.integers(0, 500, n))
    tr = branch_only(sites.tolist(), wis.tolist(), taken.tolist())
    o = oracle.compute(tr, history_len=h)
    assert_parity(run_gpu(P, tr, split=3, history_len=h), o, hist=False)          # in order across pushes
    # second half pushed first: each push sorted, the concatenation is not
    half = n // 2
    swapped = synth.Trace("swap", br=torch.cat([tr.br[half:], tr.br[:half]]).contiguous())
    assert_parity(run_gpu(P, swapped, split=2, history_len=h), oracle.compute(swapped, history_len=h), hist=False)
    assert_parity(run_gpu(P, swapped, split=2, history_len=h, on_device=False),
                  oracle.compute(swapped, history_len=h), hist=False)


def test_batch_matches_oracle_and_replays(P):
    """Invocations of uneven size, pattern and plan reduced in one batched
    graph give exactly what the oracle gives; the second call with the same
    shapes replays the cached graph."""
    from paper_1805_04207_gb300.api import compute_batch, push_trace
    traces = [synth.pattern_trace(k, c, f, seed=7, stream=i) for i, (k, c, f) in enumerate([
        ("stream", 5000, 300), ("stencil", 70_001, 9000), ("gemm", 40_000, 4096), ("zipf", 120_000, 50_000),
        ("uniform", 33_333, 33_333), ("zipf", 4096, 256)])]
    traces.append(synth.tiny())
    traces.append(synth.large(seed=8, n_mem=90_000, n_br=120_000, n_wi=40, per_wi=300, zipf_distinct=1 << 14))
    cfgs = [dict(), dict(plan=1), dict(table_slots=64), dict(history_len=31), dict(), dict(history_len=2),
            dict(), dict(plan=1, history_len=20)]
    expect = [oracle.compute(t, history_len=c.get("history_len", 16)) for t, c in zip(traces, cfgs)]
    chars = [P.Characterizer(n_opcodes=t.n_opcodes, max_work_items=1 << 24, **c) for t, c in zip(traces, cfgs)]
    try:
        for _ in range(3):
            for c, t in zip(chars, traces):
                push_trace(c, t.to("cuda"))
            got = compute_batch(chars)
            for g, o in zip(got, expect):
                assert_parity(g, o)
    finally:
        for c in chars:
            c.close()


def test_batch_of_64_with_automatic_plans(P):
    """The batched workload's shapes at oracle-sized counts: 64 invocations,
    memory events log-uniform over 2^10..2^18 and footprints over 2^6..2^16,
    patterns drawn from the five of the batched workload, every handle on the
    library's own plan choice (sort or hash plan, table size), reduced in one
    graph, twice, element by element against the oracle."""
    from paper_1805_04207_gb300.api import compute_batch, push_trace
    traces = synth.batched(64, seed=3, lo_log2=10, hi_log2=18, f_lo_log2=6, f_hi_log2=16)
    kinds = {t.meta["kind"] for t in traces}
    assert kinds == set(synth.traces.PATTERNS)
    assert min(t.n_mem for t in traces) <= (1 << 15) < max(t.n_mem for t in traces)  # both plans occur
    expect = [oracle.compute(t) for t in traces]
    chars = [P.Characterizer(n_opcodes=t.n_opcodes, max_work_items=1 << 20) for t in traces]
    dev = [t.to("cuda") for t in traces]
    try:
        for _ in range(2):
            for c, t in zip(chars, dev):
                push_trace(c, t)
            for g, o in zip(compute_batch(chars), expect):
                assert_parity(g, o)
    finally:
        for c in chars:
            c.close()


@pytest.mark.parametrize("n", [1, 2047, 2048, 2049, 64 * 2048, 64 * 2048 + 1, 65 * 2048 + 7])
def test_sort_sizes_at_tile_boundaries(P, n):
    """The radix sort's three forms -- one tile in one launch, up to 64 tiles
    with two launches per pass, more tiles with six -- at and around their
    limits: the sort plan orders the memory words, the radix path the branch
    words (events arrive out of work-item order) and the run table (runs out of
    work-item order), all compared with the oracle."""
    rng = np.random.default_rng(n)
    tr = random_trace(n, n_mem=n, n_br=n, n_wi=int(rng.integers(2, 200)), n_runs=max(1, min(n, 3000)),
                      n_ops=max(12, min(4 * n, 20000)), addr_pool=int(rng.integers(1, 5000)), n_sites=7,
                      addr_span_bits=30)
    o = oracle.compute(tr, history_len=5)
    assert_parity(run_gpu(P, tr, plan=1, history_len=5), o)
    assert_parity(run_gpu(P, tr, plan=0, history_len=5), o)


def test_deferred_pushes_give_the_same_results(P):
    """defer_pushes: device pushes recorded and ingested at compute time (in a
    batch: on parallel streams) give exactly the immediate results, also when
    host pushes of the same streams come between them (order is kept)."""
    from paper_1805_04207_gb300.api import compute_batch, push_trace
    traces = synth.batched(12, seed=5, lo_log2=10, hi_log2=17, f_lo_log2=6, f_hi_log2=14)
    expect = [oracle.compute(t) for t in traces]
    dev = [t.to("cuda") for t in traces]
    for defer in (1, 0, 1):
        chars = [P.Characterizer(n_opcodes=t.n_opcodes, max_work_items=1 << 20, defer_pushes=defer) for t in traces]
        try:
            for c, t in zip(chars, dev):
                push_trace(c, t)
            for g, o in zip(compute_batch(chars), expect):
                assert_parity(g, o)
        finally:
            for c in chars:
                c.close()
    # one handle, device and host pushes of each stream interleaved
    tr = synth.large(seed=12, n_mem=50_001, n_br=40_003, n_wi=40, per_wi=333, zipf_distinct=1 << 12)
    o = oracle.compute(tr)
    d = tr.to("cuda")
    with P.Characterizer(n_opcodes=tr.n_opcodes, defer_pushes=1) as c:
        for k, (lo, hi) in enumerate([(0, 1000), (1000, 20000), (20000, tr.n_br)]):
            c.push_branch(d.br[lo:hi].contiguous() if k != 1 else tr.br[lo:hi].contiguous())
        c.push_mem(d.mem[:30000].contiguous())
        c.push_mem(tr.mem[30000:].contiguous())
        R = tr.run_wi.shape[0]
        c.push_instr_runs(d.run_wi[:R // 2].to(torch.int32).contiguous(), d.run_off[:R // 2].contiguous(),
                          d.run_len[:R // 2].contiguous(), d.ops)
        c.push_instr_runs(tr.run_wi[R // 2:].to(torch.int32).contiguous(), tr.run_off[R // 2:].contiguous(),
                          tr.run_len[R // 2:].contiguous(), tr.ops)
        assert_parity(c.compute(), o)
        # and all device pushes, deferred to the compute
        push_trace(c, d)
        assert_parity(c.compute(), o)


@pytest.mark.parametrize("n_mem", [1 << 20, (1 << 21) + 4321])
def test_precision_fp32_compensated_within_bound(P, n_mem):
    """The FP32-compensated finalisation (c log2 c = c e + c log2 f; the first
    part exact, the second in float with Kahan compensation, FP64 only across
    threads) stays within 2^-22 bits of the FP64 oracle; counts are the same."""
    tr = synth.precision(seed=2, n_mem=n_mem, uniform_distinct=1 << 18, hot_distinct=1 << 12, n_br=1 << 16,
                         n_wi=64)
    o = oracle.compute(tr)
    g64 = run_gpu(P, tr, precision=0)
    g32 = run_gpu(P, tr, precision=1)
    assert_parity(g64, o)
    assert_parity(g32, o, entropy_tol=2.0 ** -22)
    assert abs(g32["albe"] - o["albe"]) <= 1e-6


# ---------------------------------------------------------------- partitioned invocations

def _run_partitioned(P, trace, partitions, on_device=True, **cfg):
    cfg.setdefault("n_opcodes", trace.n_opcodes)
    tr = trace.to("cuda") if on_device else trace
    with P.Characterizer(partitions=partitions, **cfg) as c:
        n = tr.n_mem
        for k in range(3):  # three pushes per stream: routing keeps push order inside each partition
            if n:
                c.push_mem(tr.mem[k * n // 3:(k + 1) * n // 3].contiguous())
            nb = tr.n_br
            if nb:
                c.push_branch(tr.br[k * nb // 3:(k + 1) * nb // 3].contiguous())
        if tr.run_wi is not None and tr.run_wi.shape[0]:
            c.push_instr_runs(tr.run_wi.to(torch.int32), tr.run_off, tr.run_len, tr.ops)
        if tr.widths is not None and tr.widths.shape[0]:
            c.push_widths(tr.widths)
        return c.compute()


@pytest.mark.parametrize("partitions", [2, 8, 64])
@pytest.mark.parametrize("on_device", [True, False])
def test_partitioned_invocation_matches_single(P, partitions, on_device):
    """Routing by superblock, site and work-item keeps every unit whole: the
    merged distributions give exactly the single invocation's metrics."""
    traces = [synth.tiny(),
              synth.large(seed=4, n_mem=300_001, n_br=120_000, n_wi=64, per_wi=300, zipf_distinct=1 << 16),
              random_trace(77, n_mem=5000, n_br=3000, n_wi=40, n_runs=200, n_ops=4000, addr_pool=900,
                           n_sites=30, addr_span_bits=24)]
    for tr in traces:
        g = _run_partitioned(P, tr, partitions, on_device)
        assert_parity(g, run_gpu(P, tr))
        assert_parity(g, oracle.compute(tr))


@pytest.mark.parametrize("plan", [1, 2])
def test_partitioned_plans_and_reuse(P, plan):
    """Both memory plans, and a handle reused for a second partitioned invocation."""
    from paper_1805_04207_gb300.api import push_trace
    tr = synth.pattern_trace("stencil", 200_000, 50_000, seed=8)
    with P.Characterizer(partitions=4, n_opcodes=tr.n_opcodes, plan=plan, table_slots=1 << 12) as c:
        for _ in range(2):
            push_trace(c, tr.to("cuda"))
            assert_parity(c.compute(want_hist=True), oracle.compute(tr))


def test_partitioned_errors(P):
    with pytest.raises(P.AiwcError):
        P.Characterizer(partitions=3)
    tr = instr_only([(0, [1, 2])], n_opcodes=8)
    with P.Characterizer(partitions=4, n_opcodes=8) as c:
        c.push_instr_runs(torch.tensor([0], dtype=torch.int32), torch.tensor([5], dtype=torch.int64),
                          torch.tensor([3], dtype=torch.int64), tr.ops)  # run past the opcode array
        with pytest.raises(P.AiwcError) as e:
            c.compute()
        assert e.value.status == P.AIWC_EINVAL
        c.push_instr_runs(tr.run_wi.to(torch.int32), tr.run_off, tr.run_len, tr.ops)  # the handle still works
        assert_parity(c.compute(want_hist=True), oracle.compute(tr))
    a = P.Characterizer(partitions=2, n_opcodes=8)
    b = P.Characterizer(n_opcodes=8)
    with pytest.raises(P.AiwcError):
        P.compute_batch([a, b])
    a.close()
    b.close()


# ---- byte-granular addresses (byte_addresses=1) ----

@pytest.mark.parametrize("seed", range(12))
def test_byte_addresses_random(P, seed):
    """Random sizes (0..255), overlapping and unaligned accesses, both memory
    plans, device and host pushes, in one and several pushes."""
    rng = np.random.default_rng(40_000 + seed)
    tr = random_trace(seed, n_mem=int(rng.integers(1, 3000)), n_br=int(rng.integers(0, 200)),
                      n_wi=int(rng.integers(1, 9)), addr_pool=int(rng.integers(1, 400)),
                      addr_span_bits=int(rng.integers(4, 40)), size_choices=[0, 1, 2, 3, 4, 8, 16, 33, 255])
    mask = int(rng.choice([0xF, 0x1, 0x6]))
    o = oracle.compute(tr, space_mask=mask, byte_addresses=1)
    g = run_gpu(P, tr, on_device=bool(seed % 2), split=1 + seed % 3, space_mask=mask, plan=seed % 3,
                byte_addresses=1)
    assert_parity(g, o)


@pytest.mark.parametrize("on_device", [True, False])
def test_byte_addresses_several_chunks(P, on_device):
    """More events than one expansion chunk (2^22) and one host staging buffer."""
    n = (1 << 22) + 4099
    rng = np.random.default_rng(5)
    addr = (1 << 34) + 4 * rng.integers(0, 1 << 22, n) + rng.integers(0, 4, n)
    sizes = rng.choice([1, 2, 4, 8], n)
    from synth import pack_mem, Trace
    mem = pack_mem(torch.from_numpy(addr), torch.from_numpy(np.arange(n) // 256), torch.from_numpy(sizes),
                   torch.from_numpy(rng.integers(0, 2, n)), torch.zeros(n, dtype=torch.int64))
    tr = Trace("bytes", mem)
    o = oracle.compute(tr, byte_addresses=1)
    assert_parity(run_gpu(P, tr, on_device=on_device, byte_addresses=1), o)


def test_byte_addresses_many_batches(P):
    """More events than one counting batch (16 chunks of 2^22): byte
    granularity equals the start-address metrics of the accesses split into
    one-byte events (the identity the oracle pins), both on the device."""
    n = (1 << 26) + 4097
    g = torch.Generator(device="cuda").manual_seed(7)
    from synth import pack_mem
    addr = (1 << 36) + 2 * torch.randint(0, 1 << 24, (n,), device="cuda", generator=g)
    sizes = torch.randint(1, 3, (n,), device="cuda", generator=g)
    wi = torch.arange(n, device="cuda") // 1024
    st = torch.randint(0, 2, (n,), device="cuda", generator=g)
    mem = pack_mem(addr, wi, sizes, st, torch.zeros_like(addr))
    with P.Characterizer(byte_addresses=1, n_opcodes=8) as c:
        c.push_mem(mem)
        got = c.compute()
    # the same accesses as one-byte events, start addresses only
    rep = torch.repeat_interleave(torch.arange(n, device="cuda"), sizes)
    first = torch.cumsum(sizes, 0) - sizes
    off = torch.arange(rep.numel(), device="cuda") - first[rep]
    one = pack_mem(addr[rep] + off, wi[rep], torch.ones_like(rep), st[rep], torch.zeros_like(rep))
    del rep, first, off
    with P.Characterizer(n_opcodes=8) as c:
        c.push_mem(one)
        want = c.compute()
    for f in ("total_reads", "total_writes", "footprint", "footprint_cover", "unique_reads", "unique_writes",
              "work_items"):
        assert got[f] == want[f], f
    assert got["entropy"] == want["entropy"]


def test_byte_addresses_large_shapes(P):
    tr = synth.large(seed=11, n_mem=500_001, n_br=0, n_wi=64, per_wi=64, zipf_distinct=1 << 16)
    for plan in (0, 1):
        assert_parity(run_gpu(P, tr, plan=plan, byte_addresses=1), oracle.compute(tr, byte_addresses=1))


def test_byte_addresses_edge_cases(P):
    # accesses of size 0 touch nothing but count their work-items
    tr = mem_only([64, 64, 4096], sizes=[0, 0, 0], wis=[3, 5, 9])
    g = run_gpu(P, tr, byte_addresses=1)
    assert (g["footprint"], g["total_reads"], g["work_items"]) == (0, 0, 3)
    assert_parity(g, oracle.compute(tr, byte_addresses=1))
    # the last byte of the domain is valid; one past it is invalid data
    edge = (1 << 61) - 2
    tr = mem_only([edge, 5], sizes=[2, 1])
    assert_parity(run_gpu(P, tr, byte_addresses=1), oracle.compute(tr, byte_addresses=1))
    with P.Characterizer(byte_addresses=1) as c:
        c.push_mem(mem_only([edge], sizes=[4]).mem.cuda())
        with pytest.raises(P.AiwcError) as ei:
            c.compute()
        assert ei.value.status == P.AIWC_EINVAL
        # the handle is reset for the next invocation
        c.push_mem(mem_only([8], sizes=[4]).mem.cuda())
        assert c.compute()["footprint"] == 4


@pytest.mark.parametrize("partitions", [2, 16])
def test_byte_addresses_partitioned(P, partitions):
    """Accesses crossing a superblock boundary are split between partitions."""
    rng = np.random.default_rng(9)
    n = 20_000
    addr = (rng.integers(0, 64, n) << 11) - rng.integers(0, 200, n) + (1 << 30)
    from synth import pack_mem, Trace
    mem = pack_mem(torch.from_numpy(addr), torch.from_numpy(rng.integers(0, 100, n)),
                   torch.from_numpy(rng.integers(0, 256, n)), torch.from_numpy(rng.integers(0, 2, n)),
                   torch.from_numpy(rng.integers(0, 2, n)))
    tr = Trace("cross", mem)
    g = _run_partitioned(P, tr, partitions, byte_addresses=1)
    assert_parity(g, oracle.compute(tr, byte_addresses=1))


# ---- branch histories per (site, work-item) (history_scope=1) ----

@pytest.mark.parametrize("seed", range(12))
def test_history_scope_random(P, seed):
    rng = np.random.default_rng(50_000 + seed)
    tr = random_trace(seed, n_mem=int(rng.integers(0, 100)), n_br=int(rng.integers(1, 3000)),
                      n_wi=int(rng.integers(1, 12)), n_sites=int(rng.integers(1, 20)))
    h = int(rng.choice([1, 2, 3, 5, 16, 20]))  # 20: longer than the per-site path takes
    o = oracle.compute(tr, history_len=h, history_scope=1)
    g = run_gpu(P, tr, on_device=bool(seed % 2), split=1 + seed % 3, history_len=h, history_scope=1,
                plan=seed % 3)
    assert_parity(g, o)


@pytest.mark.parametrize("n,n_sites,wi_sorted,h", [
    ((1 << 16) + 3, 4096, True, 3),        # site counting sort, then the global path
    (1_100_000 + 77, 4000, True, 2),
    (300_001, 50, False, 4),               # work-items out of order: radix sort
    (200_000, 5000, True, 1),              # site ids >= 4096: radix sort
])
def test_history_scope_sort_paths(P, n, n_sites, wi_sorted, h):
    """Per-site path (plan 0) and global path (plan 1) after each branch sort."""
    tr = _site_trace(11 + n_sites, n, n_sites, wi_sorted)
    o = oracle.compute(tr, history_len=h, history_scope=1)
    for split, plan in ((1, 0), (3, 0), (2, 1)):
        assert_parity(run_gpu(P, tr, split=split, history_len=h, history_scope=1, plan=plan), o)


def test_history_scope_large_shape(P):
    tr = synth.large(seed=12, n_mem=10_000, n_br=1_000_003, n_wi=1000, per_wi=1001, zipf_distinct=1 << 12)
    for h, plan in ((2, 0), (16, 0), (3, 1)):
        assert_parity(run_gpu(P, tr, history_len=h, history_scope=1, plan=plan),
                      oracle.compute(tr, history_len=h, history_scope=1))


def test_history_scope_batched_and_partitioned(P):
    from paper_1805_04207_gb300.api import compute_batch, push_trace
    traces = [_site_trace(3, 70_000, 300, True), random_trace(4, n_br=5000, n_wi=30, n_sites=40),
              synth.tiny()]
    expect = [oracle.compute(t, history_len=3, history_scope=1) for t in traces]
    chars = [P.Characterizer(n_opcodes=t.n_opcodes, history_len=3, history_scope=1) for t in traces]
    try:
        for _ in range(2):
            for c, t in zip(chars, traces):
                push_trace(c, t.to("cuda"))
            for g, o in zip(compute_batch(chars), expect):
                assert_parity(g, o)
    finally:
        for c in chars:
            c.close()
    for t, o in zip(traces, expect):
        assert_parity(_run_partitioned(P, t, 8, history_len=3, history_scope=1), o)


def test_options_in_a_batch(P):
    """Handles with byte-granular addresses and per-(site, work-item)
    histories reduced together in one batched graph, twice."""
    from paper_1805_04207_gb300.api import compute_batch, push_trace
    traces = [random_trace(61, n_mem=4000, n_br=3000, n_wi=12, n_sites=9, addr_pool=500, addr_span_bits=20,
                           size_choices=[1, 2, 4, 8, 16]),
              synth.large(seed=13, n_mem=200_001, n_br=100_000, n_wi=40, per_wi=300, zipf_distinct=1 << 14),
              synth.tiny()]
    cfgs = [dict(byte_addresses=1, history_len=2, history_scope=1), dict(byte_addresses=1),
            dict(history_scope=1, history_len=3)]
    expect = [oracle.compute(t, **c) for t, c in zip(traces, cfgs)]
    chars = [P.Characterizer(n_opcodes=t.n_opcodes, max_work_items=1 << 24, **c) for t, c in zip(traces, cfgs)]
    try:
        for _ in range(2):
            for c, t in zip(chars, traces):
                push_trace(c, t.to("cuda"))
            for g, o in zip(compute_batch(chars), expect):
                assert_parity(g, o)
    finally:
        for c in chars:
            c.close()


def test_repeated_invocations_identical(P):
    """One handle reduces the same invocation twenty times (memory and branch
    reductions on two streams at once): every result equals the oracle's and
    the first result to the bit, so no ordering between the streams leaks in."""
    tr = synth.large(seed=21, n_mem=1_000_003, n_br=400_001, n_wi=200, per_wi=500, zipf_distinct=1 << 16)
    o = oracle.compute(tr)
    from paper_1805_04207_gb300.api import push_trace
    trd = tr.to("cuda")
    with P.Characterizer(n_opcodes=tr.n_opcodes) as c:
        first = None
        for _ in range(20):
            push_trace(c, trd)
            g = c.compute()
            if first is None:
                first = g
                assert_parity(g, o)
            else:
                for k, v in first.items():
                    if k == "opcode_hist":
                        assert np.array_equal(np.asarray(g[k]), np.asarray(v))
                    elif isinstance(v, float) and math.isnan(v):
                        assert math.isnan(g[k]), k
                    else:
                        assert g[k] == v, k
