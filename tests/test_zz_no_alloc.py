"""aiwc_mem_metrics_noalloc: the entry point for callers that may not allocate
device memory (their device memory belongs to another allocator, or they must
not trigger the synchronisation that freeing memory implies). It must agree
with the regular handle-based entry point on the same events, call after call,
although every call reuses the same fixed scratch array.

Named so that pytest collects it last.
"""
from __future__ import annotations

import ctypes

import pytest
import torch

import oracle
import synth
from tests.helpers import mem_only

pytestmark = pytest.mark.gpu

MEM_FIELDS = ["total_reads", "total_writes", "footprint", "footprint_cover", "unique_reads", "unique_writes",
              "work_items"]


def _regular(P, events):
    with P.Characterizer(n_opcodes=1) as c:
        c.push_mem(events)
        return c.compute(want_hist=False)


def _noalloc(P, events, space_mask=0xF):
    stream = torch.cuda.current_stream().cuda_stream
    return P.aiwc_mem_metrics_noalloc(torch.cuda.current_device(), stream, events.data_ptr(),
                                      events.shape[0], space_mask)


def _assert_same(a, b):
    for f in MEM_FIELDS:
        assert a[f] == b[f], (f, a[f], b[f])
    for n in range(11):
        assert abs(a["entropy"][n] - b["entropy"][n]) <= 1e-9, n


def _in_range(ev):
    """The large workload's work-item ids exceed 2^20; fold them into range."""
    ev = ev.clone()
    ev[:, 1] = (ev[:, 1] & ~0xFFFFFFFF) | ((ev[:, 1] & 0xFFFFFFFF) % (1 << 20))
    return ev


def test_noalloc_matches_regular_entry_point_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_04207_gb300 as P
    traces = [synth.large(seed=21, n_mem=200_003, n_br=0, n_wi=0, per_wi=1, zipf_distinct=1 << 14),
              synth.large(seed=22, n_mem=(1 << 18), n_br=0, n_wi=0, per_wi=1, zipf_distinct=1 << 16)]
    for k, tr in enumerate(traces):
        ev = _in_range(tr.mem.cuda())
        ref = _regular(P, ev)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        got = _noalloc(P, ev)
        torch.cuda.synchronize()
        if k > 0:  # the first call may load the library's device image; later calls allocate nothing
            assert torch.cuda.mem_get_info()[0] >= free0
        _assert_same(got, ref)
        # and directly against the oracle on the same events
        _assert_same(got, oracle.compute(synth.Trace("m", mem=ev.cpu())))
        assert got["branch_events"] == 0 and got["total_instructions"] == 0
    # and once more on the first trace, after the scratch held the second one
    ev = _in_range(traces[0].mem.cuda())
    _assert_same(_noalloc(P, ev), _regular(P, ev))


def test_noalloc_recovers_after_a_failed_call_and_takes_empty_input():
    """A call that fails on its data leaves the shared scratch dirty; the next
    call must still clear everything it needs. An empty call gives zeros."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_04207_gb300 as P
    bad = mem_only([64, 128], wis=[5, 1 << 20]).mem.cuda()
    with pytest.raises(P.AiwcError) as e:
        _noalloc(P, bad)
    assert e.value.status == P.AIWC_EINVAL and "2^20" in str(e.value)
    ev = _in_range(synth.large(seed=21, n_mem=200_003, n_br=0, n_wi=0, per_wi=1, zipf_distinct=1 << 14).mem.cuda())
    _assert_same(_noalloc(P, ev), _regular(P, ev))
    empty = torch.zeros((0, 2), dtype=torch.int64, device="cuda")
    z = _noalloc(P, empty)
    assert all(z[f] == 0 for f in MEM_FIELDS) and all(x == 0.0 for x in z["entropy"])
    _assert_same(_noalloc(P, ev), _regular(P, ev))


def test_noalloc_space_mask_and_limits():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_04207_gb300 as P
    tr = mem_only([8, 8, 16, 24, 8], stores=[0, 1, 0, 1, 0], spaces=[0, 1, 1, 0, 0])
    ev = tr.mem.cuda()
    for mask in (0xF, 0x1, 0x2):
        with P.Characterizer(n_opcodes=1, space_mask=mask) as c:
            c.push_mem(ev)
            ref = c.compute(want_hist=False)
        _assert_same(_noalloc(P, ev, mask), ref)
    big = torch.zeros(((1 << 18) + 1, 2), dtype=torch.int64, device="cuda")
    with pytest.raises(P.AiwcError) as e:
        _noalloc(P, big)
    assert e.value.status == P.AIWC_EINVAL and "2^18" in str(e.value)
    raw = torch.zeros(64, dtype=torch.uint8, device="cuda")
    m = P.aiwc_metrics()
    st = P.lib.aiwc_mem_metrics_noalloc(torch.cuda.current_device(), None, raw.data_ptr() + 4, 1, 0xF,
                                        ctypes.byref(m))
    assert st == P.AIWC_EINVAL
