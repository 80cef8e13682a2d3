"""Pins for the CPU oracle against things other than itself.

* brute force: an independent pure-Python restatement (tests/brute.py) on
  hundreds of random tiny traces over small alphabets;
* closed forms from the metric definitions (Table I, Sec. III);
* hand-worked examples stored in tests/golden/hand_examples.json;
* invariants that hold at any size;
* the tiny workload's instruction and branch closed forms.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from tests import brute
from tests.helpers import branch_only, instr_only, mem_only, random_trace

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")
INT_FIELDS = ["total_instructions", "unique_opcodes", "opcode_cover", "work_items", "barriers",
              "itb_count", "itb_min", "itb_max", "itb_median_lo", "itb_median_hi",
              "ipt_count", "ipt_min", "ipt_max", "ipt_median_lo", "ipt_median_hi",
              "total_reads", "total_writes", "footprint", "footprint_cover", "unique_reads", "unique_writes",
              "branch_events", "branch_sites", "branch_cover", "branch_patterns", "branch_minsum"]


def _compare(o, b):
    for f in INT_FIELDS:
        assert o[f] == b[f], f
    assert o["itb_median"] == b["itb_median"]
    assert o["ipt_median"] == b["ipt_median"]
    assert list(o["opcode_hist"]) == list(b["opcode_hist"])
    for n in range(11):
        assert abs(o["entropy"][n] - b["entropy"][n]) <= 1e-12, n
    assert abs(o["albe"] - b["albe"]) <= 1e-15
    assert abs(o["yokota"] - b["yokota"]) <= 1e-12


@pytest.mark.parametrize("seed", range(120))
def test_oracle_matches_brute_force(seed):
    rng = np.random.default_rng(10_000 + seed)
    kw = dict(n_mem=int(rng.integers(0, 64)), n_br=int(rng.integers(0, 64)), n_wi=int(rng.integers(1, 6)),
              n_runs=int(rng.integers(1, 8)), n_ops=int(rng.integers(8, 64)), addr_pool=int(rng.integers(1, 20)),
              n_sites=int(rng.integers(1, 4)), n_opcodes=int(rng.integers(1, 7)),
              addr_span_bits=int(rng.integers(1, 16)))
    tr = random_trace(seed, **kw)
    h = int(rng.choice([1, 2, 3, 4, 16]))
    mask = int(rng.choice([0xF, 0x1, 0x3, 0xA]))
    o = oracle.compute(tr, history_len=h, space_mask=mask)
    b = brute.metrics(tr, history_len=h, space_mask=mask)
    _compare(o, b)


@pytest.mark.parametrize("num,den", [(9, 10), (1, 2), (1, 1), (1, 3)])
def test_oracle_cover_fraction_brute(num, den):
    for seed in range(20):
        tr = random_trace(500 + seed, n_mem=50, addr_pool=9)
        o = oracle.compute(tr, cover_num=num, cover_den=den)
        b = brute.metrics(tr, cover_num=num, cover_den=den)
        _compare(o, b)


def test_golden_hand_examples():
    data = json.load(open(GOLDEN))
    for ex in data["examples"]:
        if "mem" in ex:
            a, s, sp = zip(*ex["mem"])
            tr = mem_only(list(a), list(s), list(sp))
        elif "mem_repeat" in ex:
            addrs = [a for a, r in ex["mem_repeat"] for _ in range(r)]
            tr = mem_only(addrs)
        elif "br" in ex:
            st, w, t = zip(*ex["br"])
            tr = branch_only(list(st), list(w), list(t))
        elif "br_loop" in ex:
            L, P = ex["br_loop"]["length"], ex["br_loop"]["period"]
            tr = branch_only([ex["br_loop"]["site"]] * L, [0] * L, [int(j % P != P - 1) for j in range(L)])
        else:
            tr = instr_only([(w, ops) for w, ops in ex["runs"]])
        o = oracle.compute(tr, history_len=ex.get("history_len", 16))
        for k, v in ex["expect"].items():
            if k == "entropy":
                for n in range(11):
                    assert abs(o["entropy"][n] - v[n]) < 1e-6, (ex["name"], n)
            elif isinstance(v, float):
                assert abs(o[k] - v) < 1e-12, (ex["name"], k)
            else:
                assert o[k] == v, (ex["name"], k)
        for n, formula in enumerate(ex.get("entropy_formula", [])):
            exact = eval(formula, {"log2": math.log2})
            assert abs(o["entropy"][n] - exact) < 1e-14, (ex["name"], n)


@pytest.mark.parametrize("k,t", [(0, 0), (1, 0), (4, 0), (6, 2), (10, 3), (3, 5), (12, 0)])
def test_entropy_aligned_uniform_closed_form(k, t):
    """2^k addresses base + i*2^t, equally often: H_n = max(0, k - max(0, n - t))."""
    base = 1 << 40
    reps = 3
    addrs = [base + (i << t) for i in range(1 << k) for _ in range(reps)]
    o = oracle.compute(mem_only(addrs))
    for n in range(11):
        assert abs(o["entropy"][n] - max(0, k - max(0, n - t))) < 1e-12, n
    assert o["footprint"] == 1 << k
    assert o["footprint_cover"] == math.ceil(0.9 * (1 << k) - 1e-12)


def test_single_address_zero_entropy():
    o = oracle.compute(mem_only([12345] * 77, stores=[i % 2 for i in range(77)]))
    assert o["entropy"] == [0.0] * 11
    assert (o["footprint"], o["footprint_cover"], o["unique_reads"], o["unique_writes"]) == (1, 1, 1, 1)
    assert (o["total_reads"], o["total_writes"]) == (39, 38)


def test_empty_trace_all_zero():
    o = oracle.compute(synth.Trace("empty"))
    for f in INT_FIELDS:
        assert o[f] == 0, f
    assert o["entropy"] == [0.0] * 11 and o["albe"] == 0.0 and o["itb_median"] == 0.0
    assert math.isnan(o["reread_ratio"]) and math.isnan(o["unique_rw_ratio"])


def test_space_mask_filters_memory_only():
    tr = mem_only([8, 8, 16], spaces=[0, 1, 1], wis=[0, 1, 2])
    o = oracle.compute(tr, space_mask=0x1)
    assert (o["footprint"], o["total_reads"], o["work_items"]) == (1, 1, 3)


def test_branch_constant_and_alternating():
    for h in (1, 2, 16):
        for seq in ([1] * 100, [0] * 100, [j % 2 for j in range(100)]):
            o = oracle.compute(branch_only([3] * 100, [0] * 100, seq), history_len=h)
            assert o["branch_minsum"] == 0 and o["albe"] == 0.0
            assert o["branch_patterns"] == 100 - h


def test_branch_histories_are_per_site():
    # two interleaved sites, each constant: per-site histories are pure
    sites = [j % 2 for j in range(200)]
    taken = [j % 2 for j in range(200)]
    o = oracle.compute(branch_only(sites, [0] * 200, taken), history_len=4)
    assert o["branch_minsum"] == 0 and o["branch_patterns"] == 2 * (100 - 4)


def test_branch_fair_coin_bounds():
    rng = np.random.default_rng(7)
    n = 4000
    o = oracle.compute(branch_only([1] * n, [0] * n, rng.integers(0, 2, n).tolist()), history_len=2)
    assert 0.9 < o["albe"] <= 1.0


def test_itb_barrier_every_25():
    ops = []
    for k in range(100):
        ops.append(k % 8)
        if k % 25 == 24:
            ops.append(-1)
    o = oracle.compute(instr_only([(5, ops)]))
    assert (o["itb_count"], o["itb_min"], o["itb_max"], o["barriers"]) == (5, 0, 25, 4)
    assert o["itb_median"] == 25.0 and o["ipt_median"] == 100.0


def test_tiny_workload_closed_forms():
    o = oracle.compute(synth.tiny())
    # one run per work-item: 500 instructions, a barrier, then 282 (64 wi) or 281 (192 wi)
    assert (o["itb_count"], o["itb_min"], o["itb_max"]) == (512, 281, 500)
    assert (o["itb_median_lo"], o["itb_median_hi"], o["itb_median"]) == (282, 500, 391.0)
    assert (o["ipt_min"], o["ipt_max"], o["ipt_median"]) == (781, 782, 781.0)
    assert (o["total_instructions"], o["barriers"], o["work_items"]) == (200000, 256, 256)
    # 15 loop sites x 16 periods with one unpredictable exit each; N' = 16 sites x (512 - 16)
    assert (o["branch_minsum"], o["branch_patterns"], o["branch_sites"]) == (240, 16 * 496, 16)
    assert o["total_reads"] + o["total_writes"] == 65536
    # 4-byte aligned accesses: skipping 1 or 2 bits merges nothing
    assert o["entropy"][0] == o["entropy"][1] == o["entropy"][2]


@pytest.mark.parametrize("seed", range(6))
def test_invariants_medium(seed):
    tr = synth.large(seed=seed, n_mem=30_000 + 777 * seed, n_br=9_000 + 13 * seed, n_wi=17, per_wi=300,
                     zipf_distinct=1 << 14)
    o = oracle.compute(tr)
    N = o["total_reads"] + o["total_writes"]
    assert N == tr.n_mem
    H = o["entropy"]
    for n in range(10):
        assert H[n + 1] <= H[n] + 1e-12 and H[n] <= H[n + 1] + 1 + 1e-12
    assert H[0] <= math.log2(o["footprint"]) + 1e-12
    assert max(o["unique_reads"], o["unique_writes"]) <= o["footprint"] <= o["unique_reads"] + o["unique_writes"]
    assert o["itb_count"] == o["barriers"] + 17
    assert o["total_instructions"] == int(sum(o["opcode_hist"]))
    assert 0.0 <= o["albe"] <= 1.0
    coc = oracle.count_of_counts(tr.mem, 0)
    assert sum(c * m for c, m in coc.items()) == N and sum(coc.values()) == o["footprint"]


def test_memory_metrics_independent_of_event_order():
    tr = synth.large(n_mem=20_000, n_br=0, n_wi=0, per_wi=1, zipf_distinct=1 << 12)
    o1 = oracle.compute(tr)
    perm = torch.randperm(tr.n_mem, generator=torch.Generator().manual_seed(3))
    tr2 = synth.Trace("perm", mem=tr.mem[perm].contiguous())
    o2 = oracle.compute(tr2)
    for f in ["footprint", "footprint_cover", "unique_reads", "unique_writes", "total_reads", "total_writes"]:
        assert o1[f] == o2[f]
    assert max(abs(a - b) for a, b in zip(o1["entropy"], o2["entropy"])) < 1e-12


def test_invalid_inputs_rejected():
    with pytest.raises(oracle.OracleInvalidInput):
        oracle.compute(mem_only([1 << 61]))
    with pytest.raises(oracle.OracleInvalidInput):
        oracle.compute(instr_only([(0, [9])], n_opcodes=8))
    for h in (0, 32):
        with pytest.raises(oracle.OracleInvalidInput):
            oracle.compute(branch_only([0], [0], [1]), history_len=h)
    assert oracle.compute(mem_only([(1 << 61) - 1]))["footprint"] == 1


# ---------------------------------------------------------------- SIMD widths, Kiviat quantities, aggregation
# Table I SIMD rows (Sec. V records each executed instruction's result width)
# and the derived parallelism quantities of Sec. VI.

def test_simd_closed_forms():
    import statistics
    r = oracle.simd(np.full(1000, 4, dtype=np.uint16))
    assert (r["simd_count"], r["simd_max"], r["simd_sum"], r["simd_mean"], r["simd_sd"]) == (1000, 4, 4000, 4.0, 0.0)
    r = oracle.simd(np.array([1, 3] * 500, dtype=np.uint16))      # two values, equal shares
    assert (r["simd_mean"], r["simd_sd"]) == (2.0, 1.0)
    r = oracle.simd(np.zeros(0, dtype=np.uint16))
    assert (r["simd_count"], r["simd_mean"], r["simd_sd"]) == (0, 0.0, 0.0)
    rng = np.random.default_rng(5)
    w = rng.integers(0, 65536, 20_001).astype(np.uint16)
    r = oracle.simd(w)
    vals = [int(x) for x in w]
    assert r["simd_max"] == max(vals) and r["simd_sum"] == sum(vals)
    assert r["simd_sumsq"] == sum(v * v for v in vals)
    assert abs(r["simd_sd"] - statistics.pstdev(vals)) <= 1e-9 * statistics.pstdev(vals)
    assert abs(r["simd_mean"] - statistics.fmean(vals)) <= 1e-12 * statistics.fmean(vals)


def test_kiviat_quantities_on_the_tiny_workload():
    r = oracle.compute(synth.tiny())
    # 256 work-items; 256 barriers + 256 final tallies over 200,000 instructions;
    # IPT 782 (64 work-items) and 781 (192)
    assert r["granularity"] == 1.0 / 256
    assert r["barriers_per_instruction"] == 512 / 200_000
    assert r["load_imbalance"] == 1.0
    assert r["instructions_per_operand"] == 1.0 / r["simd_sum"]
    empty = oracle.compute(synth.Trace("empty"))
    assert math.isinf(empty["granularity"]) and math.isnan(empty["barriers_per_instruction"])


def test_aggregate_sum_and_median_by_hand():
    runs = [{"footprint": 5, "albe": 0.5, "entropy": [1.0, 2.0]},
            {"footprint": 1, "albe": 0.25, "entropy": [3.0, 2.0]},
            {"footprint": 9, "albe": 1.0, "entropy": [2.0, 0.0]},
            {"footprint": 2, "albe": 0.0, "entropy": [0.0, 4.0]}]
    s = oracle.aggregate(runs, "sum")
    assert s == {"footprint": 17, "albe": 1.75, "entropy": [6.0, 8.0]}
    m = oracle.aggregate(runs, "median")
    # counts: lower middle of {1, 2, 5, 9}; reals: mean of the two middle values
    assert m == {"footprint": 2, "albe": 0.375, "entropy": [1.5, 2.0]}
    m3 = oracle.aggregate(runs[:3], "median")
    assert m3 == {"footprint": 5, "albe": 0.5, "entropy": [2.0, 2.0]}


def test_library_aggregate_matches_oracle_on_cpu():
    """aiwc_aggregate is host arithmetic: it runs without a GPU."""
    P = pytest.importorskip("paper_1805_04207_gb300")
    runs = [oracle.compute(synth.pattern_trace(k, c, f, seed=2, stream=i))
            for i, (k, c, f) in enumerate([("zipf", 3000, 500), ("stencil", 4001, 900), ("stream", 2000, 300)])]
    for r in runs:
        r.pop("opcode_hist", None)
    for mode, pm in (("sum", P.AGG_SUM), ("median", P.AGG_MEDIAN)):
        g, o = P.aiwc_aggregate(runs, pm), oracle.aggregate(runs, mode)
        for k, v in o.items():
            if k == "entropy":
                assert g[k] == pytest.approx(v, rel=1e-15, abs=0)
            elif isinstance(v, float) and math.isnan(v):
                assert math.isnan(g[k])
            else:
                assert g[k] == v, k
    with pytest.raises(P.AiwcError):
        P.aiwc_aggregate(runs, 7)


# ---------------------------------------------------------------- Yokota branch entropy
# Normalisation is a reading (the paper prints none): H(history | site) / h.

def _de_bruijn(n):
    """A binary de Bruijn sequence of order n (every n-bit window once, cyclically)."""
    a, seq = [0] * (2 * n + 1), []

    def db(t, p):
        if t > n:
            if n % p == 0:
                seq.extend(a[1:p + 1])
        else:
            a[t] = a[t - p]
            db(t + 1, p)
            for j in range(a[t - p] + 1, 2):
                a[t] = j
                db(t + 1, t)
    db(1, 1)
    return seq


@pytest.mark.parametrize("h", [1, 3, 4, 7])
def test_yokota_closed_forms(h):
    s = _de_bruijn(h)
    s = s + s[:h]                      # every h-outcome window predicts exactly once
    o = oracle.compute(branch_only([5] * len(s), [0] * len(s), s), history_len=h)
    assert o["yokota"] == pytest.approx(1.0, abs=1e-12)
    const = [1] * 200                  # one history only
    assert oracle.compute(branch_only([2] * 200, [0] * 200, const), history_len=h)["yokota"] == 0.0
    # a constant site and a de Bruijn site with equal predicted counts: 1/2
    n = len(s) - h
    c = [1] * (n + h)
    tr = branch_only([1] * len(c) + [9] * len(s), [0] * (len(c) + len(s)), c + s)
    assert oracle.compute(tr, history_len=h)["yokota"] == pytest.approx(0.5, abs=1e-12)


def test_yokota_bounds_on_random_traces():
    for seed in range(30):
        tr = random_trace(seed, n_br=400, n_sites=4, n_wi=3)
        y = oracle.compute(tr, history_len=3)["yokota"]
        assert 0.0 <= y <= 1.0 + 1e-12


# ---- address granularity: every byte an access touches (byte_addresses=1) ----

def _split_into_bytes(tr):
    """The same accesses as one-byte events, one per byte touched."""
    raw = tr.mem.view(torch.uint8).reshape(-1, 16).numpy()
    rows = []
    for r in raw:
        addr = int.from_bytes(bytes(r[0:8]), "little")
        for b in range(int(r[12])):
            q = r.copy()
            q[0:8] = np.frombuffer((addr + b).to_bytes(8, "little"), dtype=np.uint8)
            q[12] = 1
            rows.append(q)
    mem = torch.from_numpy(np.array(rows, dtype=np.uint8).reshape(-1)).view(torch.int64).reshape(-1, 2) \
        if rows else torch.zeros((0, 2), dtype=torch.int64)
    return synth.Trace("bytes", mem)


@pytest.mark.parametrize("seed", range(60))
def test_byte_addresses_match_brute_force(seed):
    rng = np.random.default_rng(20_000 + seed)
    tr = random_trace(seed, n_mem=int(rng.integers(0, 48)), n_br=0, n_runs=1, n_ops=8,
                      addr_pool=int(rng.integers(1, 12)), addr_span_bits=int(rng.integers(1, 10)),
                      size_choices=[0, 1, 2, 3, 4, 8, 16])
    mask = int(rng.choice([0xF, 0x1, 0x6]))
    o = oracle.compute(tr, space_mask=mask, byte_addresses=1)
    b = brute.metrics(tr, space_mask=mask, byte_addresses=1)
    _compare(o, b)


@pytest.mark.parametrize("seed", range(20))
def test_byte_addresses_equal_one_byte_events(seed):
    """Expanding an access into its bytes is the start-address metric of one-byte events."""
    tr = random_trace(seed, n_mem=200, n_br=0, n_runs=1, n_ops=8, addr_pool=30, addr_span_bits=8,
                      size_choices=[1, 2, 4, 8, 12, 255])
    a = oracle.compute(tr, byte_addresses=1)
    s = oracle.compute(_split_into_bytes(tr), byte_addresses=0)
    for f in ("total_reads", "total_writes", "footprint", "footprint_cover", "unique_reads", "unique_writes"):
        assert a[f] == s[f], f
    assert a["entropy"] == s["entropy"]


@pytest.mark.parametrize("k", [0, 3, 8])
def test_byte_addresses_float_array_closed_form(k):
    """2^k float32 elements read once: 2^(k+2) bytes, H_n = k + 2 - n for n <= k + 2."""
    base = 1 << 32
    o = oracle.compute(mem_only([base + 4 * i for i in range(1 << k)]), byte_addresses=1)
    nb = 1 << (k + 2)
    assert (o["footprint"], o["total_reads"], o["unique_reads"]) == (nb, nb, nb)
    assert o["footprint_cover"] == math.ceil(0.9 * nb - 1e-12)
    for n in range(11):
        assert abs(o["entropy"][n] - max(0, k + 2 - n)) < 1e-12, n


def test_byte_addresses_overlap_hand_example():
    # bytes 0..3 and 2..5: counts 1,1,2,2,1,1 over 8 accesses -> H_0 = 4*(3/8) + 2*(1/4)*2 = 2.5
    o = oracle.compute(mem_only([0, 2], sizes=[4, 4]), byte_addresses=1)
    assert (o["footprint"], o["total_reads"]) == (6, 8)
    assert abs(o["entropy"][0] - 2.5) < 1e-15
    # H_1: pairs {0,1}:2, {2,3}:4, {4,5}:2 -> 1.5 bits
    assert abs(o["entropy"][1] - 1.5) < 1e-15
    assert o["entropy"][3] == 0.0


def test_byte_addresses_size_zero_and_domain():
    o = oracle.compute(mem_only([64, 64], sizes=[0, 0], wis=[3, 5]), byte_addresses=1)
    assert (o["footprint"], o["total_reads"], o["work_items"]) == (0, 0, 2)
    edge = (1 << 61) - 2
    assert oracle.compute(mem_only([edge], sizes=[4]))["footprint"] == 1
    assert oracle.compute(mem_only([edge], sizes=[2]), byte_addresses=1)["footprint"] == 2
    with pytest.raises(oracle.OracleInvalidInput):
        oracle.compute(mem_only([edge], sizes=[4]), byte_addresses=1)
    with pytest.raises(oracle.OracleInvalidInput):
        oracle.compute(mem_only([1 << 61], sizes=[0]), byte_addresses=1)


# ---- branch histories per (site, work-item) (history_scope=1) ----

@pytest.mark.parametrize("seed", range(60))
def test_per_work_item_histories_match_brute_force(seed):
    rng = np.random.default_rng(30_000 + seed)
    tr = random_trace(seed, n_mem=0, n_br=int(rng.integers(0, 80)), n_wi=int(rng.integers(1, 5)),
                      n_runs=1, n_ops=8, n_sites=int(rng.integers(1, 4)))
    h = int(rng.choice([1, 2, 3, 4]))
    o = oracle.compute(tr, history_len=h, history_scope=1)
    b = brute.metrics(tr, history_len=h, history_scope=1)
    _compare(o, b)


@pytest.mark.parametrize("seed", range(10))
def test_per_work_item_histories_equal_per_site_with_one_work_item(seed):
    tr = random_trace(seed, n_mem=0, n_br=300, n_wi=1, n_runs=1, n_ops=8, n_sites=4)
    for h in (1, 3, 16):
        a = oracle.compute(tr, history_len=h, history_scope=1)
        b = oracle.compute(tr, history_len=h, history_scope=0)
        for f in ("branch_patterns", "branch_minsum", "albe", "yokota", "branch_sites", "branch_cover"):
            assert a[f] == b[f], (h, f)


def test_per_work_item_short_sequences_predict_nothing():
    """Two outcomes per (site, work-item), as in a kernel that branches twice per thread."""
    n_wi, sites = 64, [0, 1]
    st, wi, tk = [], [], []
    for w in range(n_wi):
        for s in sites:
            for r in range(2):
                st.append(s)
                wi.append(w)
                tk.append((w + r) % 2)
    tr = branch_only(st, wi, tk)
    o = oracle.compute(tr, history_len=2, history_scope=1)
    assert (o["branch_patterns"], o["branch_minsum"], o["albe"], o["yokota"]) == (0, 0, 0.0, 0.0)
    assert o["branch_sites"] == 2
    assert oracle.compute(tr, history_len=2)["branch_patterns"] == 2 * (2 * n_wi - 2)


@pytest.mark.parametrize("h", [1, 3, 5])
def test_per_work_item_interleaved_loops_closed_form(h):
    """Two work-items each run a period-P loop at one site, pushed interleaved.

    With P = h + 1 every full per-work-item history fixes the next outcome, so
    M = 0 and N' = 2 (L - h); one history per site would mix the two loops."""
    L, P = 60, h + 1
    st, wi, tk = [], [], []
    for j in range(L):
        for w in (0, 1):
            st.append(7)
            wi.append(w)
            tk.append(int(j % P != P - 1))
    o = oracle.compute(branch_only(st, wi, tk), history_len=h, history_scope=1)
    assert (o["branch_patterns"], o["branch_minsum"]) == (2 * (L - h), 0)
    assert o["albe"] == 0.0


# ---- partitions into whole units (reading of the trace-size limit, Sec. VI) ----

def _mem_parts(mem, unit_shift: int, P: int):
    """Memory events split into P parts by a function of (space, address >> unit_shift)."""
    raw = mem.numpy().view(np.uint64).reshape(-1, 2)
    unit = (raw[:, 0] >> np.uint64(unit_shift)) * np.uint64(0x9E3779B1) + ((raw[:, 1] >> np.uint64(41)) & np.uint64(3))
    part = (unit >> np.uint64(7)) % np.uint64(P)
    return [mem[torch.from_numpy(part == p)] for p in range(P)]


@pytest.mark.parametrize("seed", range(12))
def test_partitions_into_whole_units_add_up_exactly(seed):
    """A partitioned invocation is exact because every distribution the
    metrics are taken from adds over parts made of whole units. Memory: all
    groups of skip levels 0..10 lie inside one superblock of 2^11 addresses.
    Branches: histories lie inside one site. Instructions: ITB chains lie
    inside one work-item. Checked with the oracle's exact distributions; a
    split at 2^9 addresses, which cuts skip-level-10 groups, must fail."""
    from collections import Counter
    tr = random_trace(seed, n_mem=600, n_br=400, n_wi=6, n_runs=16, n_ops=300, addr_pool=200, n_sites=6,
                      addr_span_bits=16)
    P = 4
    whole = oracle.compute(tr, history_len=2)
    parts = _mem_parts(tr.mem, 11, P)
    for n in range(11):
        summed = Counter()
        for m in parts:
            summed.update(oracle.count_of_counts(m, n))
        assert dict(summed) == oracle.count_of_counts(tr.mem, n), n
    pm = [oracle.compute(synth.Trace("m", m), history_len=2) for m in parts]
    for f in ("total_reads", "total_writes", "footprint", "unique_reads", "unique_writes"):
        assert sum(o[f] for o in pm) == whole[f], f
    # branches by site, in both history scopes
    raw = tr.br.numpy().view(np.uint64)
    site = raw & np.uint64(0xFFFFFFFF)
    for scope in (0, 1):
        ws = oracle.compute(tr, history_len=2, history_scope=scope)
        pb = [oracle.compute(synth.Trace("b", br=tr.br[torch.from_numpy(site % np.uint64(P) == p)]), history_len=2,
                             history_scope=scope) for p in range(P)]
        for f in ("branch_events", "branch_sites", "branch_patterns", "branch_minsum"):
            assert sum(o[f] for o in pb) == ws[f], (scope, f)
        # the Yokota numerator, N' h H(history | site), adds over sites
        num = sum(o["yokota"] * o["branch_patterns"] for o in pb)
        assert abs(num - ws["yokota"] * ws["branch_patterns"]) <= 1e-9 * max(1.0, num), scope
    # instructions by work-item
    wi = tr.run_wi.numpy()
    pi = []
    for p in range(P):
        sel = np.nonzero(wi % P == p)[0]
        runs = [(int(wi[r]), tr.ops[int(tr.run_off[r]):int(tr.run_off[r] + tr.run_len[r])].tolist()) for r in sel]
        pi.append(oracle.compute(instr_only(runs, n_opcodes=tr.n_opcodes)) if runs else None)
    pi = [o for o in pi if o is not None]
    for f in ("total_instructions", "barriers", "itb_count", "ipt_count"):
        assert sum(o[f] for o in pi) == whole[f], f
    assert min(o["itb_min"] for o in pi) == whole["itb_min"] and max(o["itb_max"] for o in pi) == whole["itb_max"]
    assert (np.sum([o["opcode_hist"] for o in pi], axis=0) == whole["opcode_hist"]).all()


def test_partitions_that_cut_groups_do_not_add_up():
    """The control: parts of 2^9 addresses cut skip-level-10 groups, and the
    summed distribution differs from the whole's for some trace."""
    from collections import Counter
    differs = False
    for seed in range(6):
        tr = random_trace(seed, n_mem=600, n_br=0, n_runs=1, n_ops=8, addr_pool=200, addr_span_bits=16)
        summed = Counter()
        for m in _mem_parts(tr.mem, 9, 4):
            summed.update(oracle.count_of_counts(m, 10))
        differs |= dict(summed) != oracle.count_of_counts(tr.mem, 10)
    assert differs


@pytest.mark.parametrize("seed", range(8))
def test_byte_accesses_split_at_a_superblock_edge_are_unchanged(seed):
    """With byte-granular addresses an access is the set of bytes it touches,
    so cutting one that crosses a 2^11-address boundary into two accesses
    (how a partitioned invocation routes it) changes no metric."""
    rng = np.random.default_rng(seed)
    n = 300
    edge = (rng.integers(1, 6, n) << 11).astype(np.int64)
    addr = edge - rng.integers(0, 12, n)           # start up to 12 bytes before an edge
    size = rng.integers(0, 17, n)
    st, sp, wi = rng.integers(0, 2, n), rng.integers(0, 4, n), rng.integers(0, 5, n)
    tr = mem_only(addr.tolist(), st.tolist(), sp.tolist(), wi.tolist(), size.tolist())
    a2, s2, st2, sp2, wi2 = [], [], [], [], []
    for i in range(n):
        cut = max(0, min(int(size[i]), int(edge[i] - addr[i])))
        pieces = [(int(addr[i]), cut), (int(edge[i]), int(size[i]) - cut)] if 0 < cut < size[i] else \
            [(int(addr[i]), int(size[i]))]
        for a, s in pieces:
            a2.append(a)
            s2.append(s)
            st2.append(int(st[i]))
            sp2.append(int(sp[i]))
            wi2.append(int(wi[i]))
    split = mem_only(a2, st2, sp2, wi2, s2)
    assert len(a2) > n  # some accesses did cross
    o, b = oracle.compute(tr, byte_addresses=1), oracle.compute(split, byte_addresses=1)
    for f in ("total_reads", "total_writes", "footprint", "footprint_cover", "unique_reads", "unique_writes",
              "work_items"):
        assert o[f] == b[f], f
    assert o["entropy"] == b["entropy"]


def entropy_from_coc(coc: dict) -> float:
    """H = log2 N - (1/N) sum_c m_c c log2 c (Table I memory entropy under reading R1)."""
    N = sum(c * m for c, m in coc.items())
    if N == 0:
        return 0.0
    return math.log2(N) - math.fsum(m * c * math.log2(c) for c, m in coc.items()) / N


def colliding_spaces_trace(seed: int) -> "synth.Trace":
    """Accesses in all four address spaces whose numeric addresses repeat
    across spaces, at several alignments, so that dropping the space tag or
    the skip shift changes the grouping."""
    rng = np.random.default_rng(seed)
    pool = np.concatenate([rng.integers(0, 1 << 13, 24), (rng.integers(0, 64, 8) << 6)]).astype(np.int64)
    n = 3000
    addr = pool[rng.integers(0, pool.size, n)]
    space = rng.integers(0, 4, n)
    store = rng.integers(0, 2, n)
    return mem_only(addr.tolist(), store.tolist(), space.tolist())


@pytest.mark.parametrize("seed", range(3))
def test_count_of_counts_gives_every_entropy(seed):
    """The helper's m_c at skip level n must reproduce the oracle's entropy[n]
    for every n = 0..10, on every space mask: the helper forms its groups
    (space tag, address >> n) on its own, so a slip in it shows here."""
    tr = colliding_spaces_trace(seed)
    for mask in (0xF, 0x5, 0x2):
        o = oracle.compute(tr, space_mask=mask)
        for n in range(11):
            coc = oracle.count_of_counts(tr.mem, n, space_mask=mask)
            assert sum(c * m for c, m in coc.items()) == o["total_reads"] + o["total_writes"]
            assert abs(entropy_from_coc(coc) - o["entropy"][n]) <= 1e-12, (mask, n)
        assert sum(oracle.count_of_counts(tr.mem, 0, space_mask=mask).values()) == o["footprint"]
