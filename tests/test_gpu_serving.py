"""Serving: jobs streaming their traces in chunks through a server with a
bounded number of slots and an HBM budget. Every job's metrics must be the
same in the mix as when it runs alone, and the same as the oracle's."""
from __future__ import annotations

import pytest
import torch

import oracle
import synth
from tests.test_gpu_parity import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_04207_gb300 as P
    return P


def _traces():
    out = [synth.pattern_trace(k, c, f, seed=31, stream=i) for i, (k, c, f) in enumerate([
        ("zipf", 200_000, 60_000), ("stencil", 150_001, 20_000), ("stream", 9_000, 700), ("gemm", 64_000, 16_384),
        ("uniform", 100_000, 90_000), ("zipf", 5_000, 300), ("stencil", 300_000, 100_000)])]
    out.append(synth.tiny())
    out.append(synth.large(seed=9, n_mem=250_000, n_br=90_000, n_wi=50, per_wi=400, zipf_distinct=1 << 15))
    return out


def _push_chunks(job, tr, n_chunks=4):
    tr = tr.to("cuda")
    n = tr.n_mem
    for k in range(n_chunks):
        part = tr.mem[k * n // n_chunks:(k + 1) * n // n_chunks].contiguous()
        if part.shape[0]:
            job.push_mem(part)
    b = tr.n_br
    for k in range(2):
        part = tr.br[k * b // 2:(k + 1) * b // 2].contiguous()
        if part.shape[0]:
            job.push_branch(part)
    job.push_instr_runs(tr.run_wi.to(torch.int32), tr.run_off, tr.run_len, tr.ops)
    if tr.widths is not None and tr.widths.shape[0]:
        job.push_widths(tr.widths)


def test_serving_results_equal_alone_and_in_the_mix(P):
    from paper_1805_04207_gb300.serving import Server
    traces = _traces()
    cfg = dict(max_work_items=1 << 24, table_slots=1 << 16)
    alone = [P.characterize(t.to("cuda"), n_opcodes=t.n_opcodes, **cfg) for t in traces]
    with Server(max_jobs=3, workers=2, hbm_budget=6 << 30) as srv:
        pending = list(range(len(traces)))
        running, results = {}, {}
        while pending or running:
            while pending:
                i = pending[0]
                job = srv.open(1 << 30, n_opcodes=traces[i].n_opcodes, **cfg)
                if job is None:
                    break  # no slot or budget: retry once a job completes
                _push_chunks(job, traces[i])
                job.finish()
                running[i] = job
                pending.pop(0)
            for i, job in list(running.items()):
                r = job.poll(want_hist=True)
                if r is not None:
                    results[i] = r
                    del running[i]
        st = srv.stats()
    assert st["admitted"] == len(traces) and st["completed"] == len(traces)
    assert st["rejected"] > 0  # three slots for nine jobs: some had to wait
    for i, t in enumerate(traces):
        assert_parity(results[i], alone[i])
        if t.n_mem <= 300_000:
            assert_parity(results[i], oracle.compute(t))


def test_serving_admission_limits(P):
    from paper_1805_04207_gb300.serving import Server
    with Server(max_jobs=2, workers=1, hbm_budget=1 << 30) as srv:
        with pytest.raises(P.AiwcError) as e:
            srv.open(2 << 30)
        assert e.value.status == P.AIWC_ENOMEM
        a = srv.open(400 << 20, max_work_items=1 << 20, table_slots=1 << 12, n_opcodes=64)
        b = srv.open(400 << 20, max_work_items=1 << 20, table_slots=1 << 12)
        assert a is not None and b is not None
        assert srv.open(100 << 20, max_work_items=1 << 20) is None  # no slot left
        tr = synth.tiny()
        _push_chunks(a, tr)
        r = a.wait(want_hist=True)
        assert_parity(r, oracle.compute(tr))
        assert srv.open(700 << 20, max_work_items=1 << 20) is None  # 400 MiB still reserved by b
        b.finish()
        b.wait()
        c = srv.open(700 << 20, max_work_items=1 << 20, table_slots=1 << 12)
        assert c is not None
        c.wait()


def test_serving_job_options_are_honoured(P):
    """A slot's handle is reused only by a job with the same metric options:
    jobs that switch byte-granular addresses and history scope on and off in
    one slot each get their own options' results."""
    from paper_1805_04207_gb300.serving import Server
    from tests.helpers import random_trace
    tr = random_trace(5, n_mem=3000, n_br=3000, n_wi=8, n_sites=5, addr_pool=300, addr_span_bits=14,
                      size_choices=[1, 2, 4, 8])
    with Server(max_jobs=1, workers=1, hbm_budget=2 << 30) as srv:
        for opts in (dict(), dict(byte_addresses=1), dict(history_scope=1), dict(byte_addresses=1, history_scope=1),
                     dict()):
            job = srv.open(256 << 20, n_opcodes=tr.n_opcodes, history_len=3, max_work_items=1 << 20,
                           table_slots=1 << 12, **opts)
            assert job is not None
            _push_chunks(job, tr)
            r = job.wait(want_hist=True)
            assert_parity(r, oracle.compute(tr, history_len=3, **opts))
