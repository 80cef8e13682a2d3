"""Plant plausible mistakes in a copy of the oracle and check that the pins catch each.

Every mutation below is a one-line slip of the kind the pins exist for (a
dropped term, an off-by-one, a wrong bit, a missing tag). The edited copy is
compiled on the CPU into a temporary directory; the real oracle is untouched.
"""
from __future__ import annotations

import json
import math
import os
import statistics

import numpy as np
import pytest
import torch

import oracle
import synth
from tests import brute
from tests.helpers import branch_only, instr_only, mem_only, random_trace
from tests.test_oracle_pins import GOLDEN, INT_FIELDS, colliding_spaces_trace, entropy_from_coc

MUTATIONS = {
    "history_skips_one_more": ("for (size_t j = h; j < seq.size(); ++j)", "for (size_t j = h + 1; j < seq.size(); ++j)"),
    "history_in_push_order": ("std::stable_sort(seq.begin(), seq.end(),", "if (0) std::stable_sort(seq.begin(), seq.end(),"),
    "no_space_tag": ("uint64_t key = ((uint64_t)space << 61) | (addr + b);", "uint64_t key = addr + b;"),
    "bytes_one_short": ("const uint64_t touched = cfg->byte_addresses ? size : 1;",
                        "const uint64_t touched = cfg->byte_addresses ? (size ? size - 1 : 0) : 1;"),
    "bytes_all_at_start": ("uint64_t key = ((uint64_t)space << 61) | (addr + b);",
                           "uint64_t key = ((uint64_t)space << 61) | addr;"),
    "bytes_size0_counts_one": ("const uint64_t touched = cfg->byte_addresses ? size : 1;",
                               "const uint64_t touched = cfg->byte_addresses ? (size ? size : 1) : 1;"),
    "bytes_domain_unchecked": ("if (cfg->byte_addresses && size > 0 && addr + size - 1 >= kAddrLimit) return 1;",
                               "if (0) return 1;"),
    "per_wi_history_not_split": ("for (auto& e : seq) per_wi[e.first].push_back(e.second);",
                                 "for (auto& e : seq) per_wi[0].push_back(e.second);"),
    "per_wi_patterns_keyed_by_wi": ("for (auto& w : per_wi) predict(kv.first, w.second);",
                                    "for (auto& w : per_wi) predict(kv.first ^ (w.first << 8), w.second);"),
    "skip_inner_off_by_one": ("while (j < n_acc && (all_keys[j] >> n) == g) ++j;",
                              "while (j < n_acc && (all_keys[j] >> (n + 1)) == (g >> 1)) ++j;"),
    "cover_strict": ("if ((unsigned __int128)den * cum >= (unsigned __int128)num * total) return k + 1;",
                     "if ((unsigned __int128)den * cum > (unsigned __int128)num * total) return k + 1;"),
    "median_upper_only": ("*med = 0.5 * ((double)*lo + (double)*hi);", "*med = (double)*hi;"),
    "no_trailing_itb": ("    itb.push_back(kv.second.first);\n", "\n"),
    "entropy_unweighted": ("acc.add(-p * std::log2(p));", "acc.add(-std::log2(p));"),
    "store_bit_wrong": ("if (flags & 1u) write_keys.push_back(key);", "if (flags & 2u) write_keys.push_back(key);"),
    "minsum_max": ("minsum += std::min(t, n - t);", "minsum += std::max(t, n - t);"),
    "history_includes_outcome": ("for (size_t k = j - h; k < j; ++k)", "for (size_t k = j - h + 1; k <= j; ++k)"),
    "barrier_counted_as_instruction": ("        itb.push_back(st.first);\n        st.first = 0;\n        ++barriers;",
                                       "        itb.push_back(st.first);\n        st.first = 0;\n        ++barriers;\n        ++hist[0];"),
    "work_items_memory_ignored": ("    work_items.insert(wi);\n    if (addr", "    if (addr"),
    "yokota_site_term_dropped": ("site_sum.add(n * std::log2(n));", "site_sum.add(0.0 * n);"),
    "yokota_not_per_bit": ("((double)npat * (double)h)", "((double)npat)"),
    "simd_square_dropped": ("q += w * w;", "q += w;"),
    "simd_max_first_only": ("if (w > m) m = w;", "if (i == 0) m = w;"),
    "space_mask_ignored": ("if (!((cfg->space_mask >> space) & 1u)) continue;", "if (0) continue;"),
    "unique_writes_are_unique_reads": (
        "out->unique_writes = std::unique(write_keys.begin(), write_keys.end()) - write_keys.begin();",
        "out->unique_writes = out->unique_reads;"),
    "branch_cover_over_predicted": ("site_counts.push_back(seq.size());",
                                    "site_counts.push_back(seq.size() > h ? seq.size() - h : 0);"),
    "ipt_counts_barriers": ("        itb.push_back(st.first);\n        st.first = 0;\n        ++barriers;",
                            "        itb.push_back(st.first);\n        st.first = 0;\n        ++barriers;\n        ++st.second;"),
    "reread_ratio_inverted": ("out->reread_ratio = (double)out->unique_reads / (double)out->total_reads;",
                              "out->reread_ratio = (double)out->total_reads / (double)out->unique_reads;"),
    "coc_no_space_tag": ("keys.push_back((((uint64_t)space << 61) | addr) >> n);", "keys.push_back(addr >> n);"),
    "coc_skip_ignored": ("keys.push_back((((uint64_t)space << 61) | addr) >> n);",
                         "keys.push_back(((uint64_t)space << 61) | addr);"),
    "coc_space_mask_ignored": ("if (!((space_mask >> space) & 1u)) continue;", "if (0) continue;"),
    "coc_group_counted_twice": ("coc[j - i] += 1;", "coc[j - i] += 1 + (j - i > 1);"),
    "cover_fraction_swapped": (
        "if ((unsigned __int128)den * cum >= (unsigned __int128)num * total) return k + 1;",
        "if ((unsigned __int128)num * cum >= (unsigned __int128)den * total) return k + 1;"),
}


def _pins_pass(lib):
    """A compact run of the oracle pins against the library at `lib`."""
    def comp(tr, **kw):
        return oracle.compute(tr, lib_path=lib, **kw)
    try:
        for seed in range(40):
            rng = np.random.default_rng(10_000 + seed)
            tr = random_trace(seed, n_mem=int(rng.integers(0, 64)), n_br=int(rng.integers(0, 64)),
                              n_wi=int(rng.integers(1, 6)), n_runs=int(rng.integers(1, 8)),
                              n_ops=int(rng.integers(8, 64)), addr_pool=int(rng.integers(1, 20)),
                              n_sites=int(rng.integers(1, 4)), addr_span_bits=int(rng.integers(1, 16)))
            h = int(rng.choice([1, 2, 3]))
            mask = 0xF if seed % 2 else int(rng.choice([0x1, 0x3, 0xA]))
            o, b = comp(tr, history_len=h, space_mask=mask), brute.metrics(tr, history_len=h, space_mask=mask)
            for f in INT_FIELDS:
                if o[f] != b[f]:
                    return False
            if o["itb_median"] != b["itb_median"] or o["ipt_median"] != b["ipt_median"]:
                return False
            if list(o["opcode_hist"]) != list(b["opcode_hist"]):
                return False
            if max(abs(x - y) for x, y in zip(o["entropy"], b["entropy"])) > 1e-12:
                return False
            if abs(o["yokota"] - b["yokota"]) > 1e-12 or abs(o["albe"] - b["albe"]) > 1e-15:
                return False
        for ex in json.load(open(GOLDEN))["examples"]:
            if "mem" in ex:
                a, s, sp = zip(*ex["mem"])
                tr = mem_only(list(a), list(s), list(sp))
            elif "mem_repeat" in ex:
                tr = mem_only([a for a, r in ex["mem_repeat"] for _ in range(r)])
            elif "br" in ex:
                st, w, t = zip(*ex["br"])
                tr = branch_only(list(st), list(w), list(t))
            elif "br_loop" in ex:
                L, P = ex["br_loop"]["length"], ex["br_loop"]["period"]
                tr = branch_only([ex["br_loop"]["site"]] * L, [0] * L, [int(j % P != P - 1) for j in range(L)])
            else:
                tr = instr_only([(w, ops) for w, ops in ex["runs"]])
            o = comp(tr, history_len=ex.get("history_len", 16))
            for k, v in ex["expect"].items():
                if k == "entropy":
                    if max(abs(o["entropy"][n] - v[n]) for n in range(11)) > 1e-6:
                        return False
                elif abs(o[k] - v) > 1e-12:
                    return False
        # the count-of-counts helper reproduces every entropy level on every space mask
        for seed in range(2):
            tr = colliding_spaces_trace(seed)
            for mask in (0xF, 0x5):
                o = comp(tr, space_mask=mask)
                for n in range(11):
                    coc = oracle.count_of_counts(tr.mem, n, space_mask=mask, lib_path=lib)
                    if abs(entropy_from_coc(coc) - o["entropy"][n]) > 1e-12:
                        return False
        o = comp(synth.tiny())
        if (o["itb_median"], o["branch_minsum"], o["branch_patterns"]) != (391.0, 240, 7936):
            return False
        # SIMD widths: a two-value closed form and a brute-force population SD
        tr = instr_only([(0, [1, 2])])
        tr.widths = torch.tensor([1, 3] * 50 + [7], dtype=torch.int16)
        o = comp(tr)
        vals = [1, 3] * 50 + [7]
        if (o["simd_max"], o["simd_sum"], o["simd_sumsq"]) != (7, sum(vals), sum(v * v for v in vals)):
            return False
        if abs(o["simd_sd"] - statistics.pstdev(vals)) > 1e-12:
            return False
        for k, t in ((4, 0), (6, 2)):
            o = comp(mem_only([(1 << 40) + (i << t) for i in range(1 << k) for _ in range(3)]))
            if max(abs(o["entropy"][n] - max(0, k - max(0, n - t))) for n in range(11)) > 1e-12:
                return False
        # byte addresses: brute force on random sizes, and the overlap hand example
        for seed in range(12):
            tr = random_trace(seed, n_mem=40, n_br=0, n_runs=1, n_ops=8, addr_pool=8, addr_span_bits=6,
                              size_choices=[0, 1, 2, 4, 8])
            o, b = comp(tr, byte_addresses=1), brute.metrics(tr, byte_addresses=1)
            if any(o[f] != b[f] for f in INT_FIELDS):
                return False
            if max(abs(x - y) for x, y in zip(o["entropy"], b["entropy"])) > 1e-12:
                return False
        o = comp(mem_only([0, 2], sizes=[4, 4]), byte_addresses=1)
        if (o["footprint"], o["total_reads"]) != (6, 8) or abs(o["entropy"][0] - 2.5) > 1e-15:
            return False
        # a last byte outside the 61-bit domain is invalid data
        try:
            comp(mem_only([(1 << 61) - 2], sizes=[4]), byte_addresses=1)
            return False
        except oracle.OracleInvalidInput:
            pass
        # per-(site, work-item) histories: brute force and the interleaved-loop closed form
        for seed in range(12):
            tr = random_trace(seed, n_mem=0, n_br=60, n_wi=3, n_runs=1, n_ops=8, n_sites=2)
            o, b = comp(tr, history_len=2, history_scope=1), brute.metrics(tr, history_len=2, history_scope=1)
            if any(o[f] != b[f] for f in INT_FIELDS) or abs(o["yokota"] - b["yokota"]) > 1e-12:
                return False
        st = [7] * 120
        wi = [j % 2 for j in range(120)]
        tk = [int((j // 2) % 4 != 3) for j in range(120)]
        o = comp(branch_only(st, wi, tk), history_len=3, history_scope=1)
        if (o["branch_patterns"], o["branch_minsum"]) != (2 * (60 - 3), 0):
            return False
    except (oracle.OracleInvalidInput, ValueError):  # a mutated oracle may also fail outright
        return False
    return True


def test_unmodified_oracle_passes(tmp_path):
    lib = oracle.build_variant(oracle.source(), str(tmp_path), "clean")
    assert _pins_pass(lib)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = oracle.source()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    lib = oracle.build_variant(src.replace(old, new), str(tmp_path), name)
    assert not _pins_pass(lib), f"pins did not catch planted mistake {name}"
