#!/usr/bin/env python3
"""Throughput of the AIWC trace reduction on GB300.

A step is one kernel invocation reduced end to end: push the memory, branch
and instruction streams and compute every Table I metric. The workload is the
large invocation (2^28 memory events mixing a 7-point stencil over 256^3,
16x16-tiled SGEMM accesses for 2048^3 and Zipf(1.05) gathers over 2^26
addresses; 2^26 branch events over 4,096 sites; 2^30 opcodes over 256 ids),
generated on the device from a seed. Metric: memory events characterised per
second (all metrics computed), whole job.

`python bench.py [--gpus N --steps K --warmup W] [--impl reference]`; for N > 1
launch one process per GPU with torch.distributed.run (replicas: each rank
reduces its own invocation, no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "memory events/s characterized (all AIWC metrics)"
UNIT = "events/s"
WORKLOAD = ("large invocation: 2^28 memory events (stencil 256^3 + tiled SGEMM 2048^3 + Zipf(1.05) over 2^26), "
            "2^26 branch events over 4096 sites, 2^30 opcodes over 256 ids")
# Algorithmic bytes per unit (read once): 16 B per memory event, 8 B per
# branch event, 2 B per opcode; plus 16 B per distinct address and 8 B per
# history pattern for the run tables the method must form. A sort stage is
# credited with one read and one write of each 8-byte key it orders.
ALG_BYTES = {"mem_event": 16, "branch_event": 8, "opcode": 2, "distinct_key": 16, "pattern": 8}
KERNEL_FILES = {"mem_ingest": "mem.cu", "branch_ingest": "branch.cu", "instr_runs": "instr.cu", "mem_sort": "sort.cu",
                "mem_scatter": "mem_hash.cu", "mem_levels": "mem_hash.cu", "branch_sort": "branch.cu", "windows": "branch.cu", "pattern_sort": "sort.cu",
                "pattern_runs": "branch.cu", "run_sort": "sort.cu", "run_combine": "instr.cu",
                "finalize": "finalize.cu", "mem_expand": "mem.cu"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=0, help="shrink the workload by 2^scale (testing only)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="large", choices=["large", "batched", "serving", "precision", "partitioned"],
                    help="large (default): the 2^28-event invocation; batched: 512 uneven invocations per "
                         "step in one graph; serving: Poisson jobs streaming chunks; precision: 2^30 events, "
                         "FP32-compensated vs FP64 entropies")
    ap.add_argument("--jobs", type=int, default=100, help="serving: number of jobs")
    ap.add_argument("--partitions", type=int, default=8, help="partitioned: number of partitions")
    ap.add_argument("--byte-addresses", action="store_true",
                    help="large: every byte an access touches is an access (about 5 one-byte accesses per event)")
    ap.add_argument("--history-scope", type=int, default=0, choices=[0, 1],
                    help="large: 1 = one branch history per (site, work-item)")
    return ap.parse_args()


def options(args) -> dict:
    """Handle options of the large workload's variants."""
    o = {}
    if args.byte_addresses:
        o["byte_addresses"] = 1
    if args.history_scope:
        o["history_scope"] = 1
    return o


def workload_name(args) -> str:
    w = WORKLOAD
    if args.byte_addresses:
        w += "; byte-granular addresses (every byte an access touches is an access)"
    if args.history_scope:
        w += "; branch histories per (site, work-item)"
    return w


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.lines = []
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def source_sha(fname: str) -> str:
    h = hashlib.sha256()
    for f in (fname, "aiwc_internal.cuh", "runs.cuh", "common.cuh"):
        p = os.path.join(ROOT, "paper_1805_04207_gb300", "csrc", f)
        if os.path.exists(p):
            h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def traffic_for(stage: str):
    """DRAM bytes per launch of a stage from the committed ncu summary, if the
    kernel source still matches the one the counters were taken on."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p)).get(stage)
    except Exception:
        return None
    if not d or d.get("source_sha") != source_sha(KERNEL_FILES.get(stage, "")):
        return None
    return d.get("dram_bytes_per_step")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _oracle_sample(scale_shift: int, opts: dict, seed: int):
    """A bounded, large-shaped sample for the oracle: (trace, n_mem, n_br, n_wi)."""
    import synth
    if opts.get("byte_addresses"):
        scale_shift += 3  # about five one-byte accesses per event
    n_mem = 1 << (26 - scale_shift)
    n_br = 1 << (24 - scale_shift)
    n_wi = max(1, 1 << (18 - scale_shift))
    tr = synth.large(seed=seed, n_mem=n_mem, n_br=n_br, n_wi=n_wi, per_wi=1024,
                     zipf_distinct=1 << (24 - scale_shift))
    return tr, n_mem, n_br, n_wi, scale_shift


def cpu_baseline(scale_shift: int, opts=None):
    """The oracle, as it stands, on a bounded sample of the same workload."""
    import oracle
    opts = opts or {}
    tr, n_mem, n_br, n_wi, sh = _oracle_sample(scale_shift, opts, 0)
    t0 = time.perf_counter()
    oracle.compute(tr, **opts)
    dt = time.perf_counter() - t0
    return {"value": n_mem / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"large-shaped sample: {n_mem} memory, {n_br} branch, {n_wi * 1024} opcodes "
                      f"(Zipf over 2^{24 - sh}), single-threaded C++ oracle, {dt:.1f} s"}, dt


def _oracle_replica(job):
    """One process of the all-cores baseline: build its own sample, wait for
    every replica, then time the oracle on it (wall clock of this host)."""
    scale_shift, opts, seed, barrier = job
    import oracle
    tr, n_mem, _, _, _ = _oracle_sample(scale_shift, opts, seed)
    barrier.wait(timeout=600)
    t0 = time.time()
    oracle.compute(tr, **opts)
    return n_mem, t0, time.time()


def cpu_baseline_all_cores(scale_shift: int, opts=None, procs: int = 0):
    """The oracle, as it stands, as independent replicas on every host core:
    one process per core, each reducing its own sample (seed = its index),
    all started together. Throughput = all samples' events / the span from
    the first start to the last finish."""
    import multiprocessing as mp
    opts = opts or {}
    if not procs:
        procs = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    ctx = mp.get_context("spawn")  # the parent may hold a CUDA context: never fork
    with ctx.Manager() as man:
        barrier = man.Barrier(procs)
        with ctx.Pool(procs) as pool:
            # a bounded wait: a replica that dies must not hang the benchmark
            res = pool.map_async(_oracle_replica,
                                 [(scale_shift, opts, seed, barrier) for seed in range(procs)]).get(timeout=900)
    n = sum(r[0] for r in res)
    span = max(r[2] for r in res) - min(r[1] for r in res)
    return {"value": n / span, "unit": UNIT, "cores": procs, "kind": "oracle replicas",
            "sample": f"{procs} processes, each the single-threaded C++ oracle on its own large-shaped sample "
                      f"of {res[0][0]} memory events; {span:.2f} s from the first start to the last finish"}


def run_reference(args, rank, world):
    """The reference arm: the oracle, as it stands, on the host cores. Every
    one of the --warmup + --steps steps reduces the same bounded sample of the
    large workload (2^23 memory events of the same shapes, sized so that the
    whole run takes a minute or so); the line reports the steps it ran and the
    time per sample step."""
    if rank != 0:
        return
    if args.workload != "large":
        print(json.dumps({"impl": "reference", "unavailable": f"the reference arm (the oracle on the host cores) "
                          f"times the large invocation only, not the {args.workload} workload"}), flush=True)
        return
    import oracle
    oracle.build()
    opts = options(args)
    tr, n_mem, n_br, n_wi, sh = _oracle_sample(args.scale + 3, opts, 0)
    for _ in range(args.warmup):
        oracle.compute(tr, **opts)
    dts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.compute(tr, **opts)
        dts.append(time.perf_counter() - t0)
    step_s = sum(dts) / len(dts)
    v = n_mem / step_s
    sample = (f"{n_mem} memory, {n_br} branch, {n_wi * 1024} opcode events of the large invocation's shapes "
              f"(Zipf over 2^{24 - sh}) per step")
    workload = f"{workload_name(args)}; reference sample per step: {sample}"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * step_s, 3),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64+f64", "data": "synthetic",
            "config": {"workload": workload, "seed": 0, "inputs": "host memory (the oracle runs on the CPU)",
                       "parallelism": "one host core", "scale_shift": args.scale, **opts},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{sample}; single-threaded C++ oracle, {args.steps} timed steps of "
                                       f"{step_s:.2f} s"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks (the slowest replica sets the job's time)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


L2_BYTES = 129 << 20


def inputs_note(n_bytes: int) -> str:
    """How the timed inputs relate to L2: above it no flush is needed between
    steps; at or below it (small test scales only) the note says so."""
    rel = "> L2 (no flush)" if n_bytes > L2_BYTES else "<= L2 (test scale: L2-resident between steps)"
    return f"device-resident, {n_bytes / 1e9:.2f} GB {rel}"


def replica_throughput(units_per_rank: int, world: int, seconds: float) -> float:
    """Whole-job throughput of `world` replicas each processing units_per_rank."""
    return world * units_per_rank / seconds


def base_line(args, world, value, ms, extra):
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": round(ms, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64+f64", "data": "synthetic", "impl": "ours"}
    line.update(extra)
    return line


def run_batched(args, P, torch, local, world, rank):
    import synth
    from paper_1805_04207_gb300.api import compute_batch, push_trace
    traces = synth.batched(512, device="cuda", seed=rank)
    n_mem = sum(t.n_mem for t in traces)
    # device pushes are deferred to the batched compute, which ingests the
    # invocations side by side
    chars = [P.Characterizer(device=local, n_opcodes=t.n_opcodes, max_work_items=1 << 20, defer_pushes=1)
             for t in traces]
    for t in traces:
        t.run_wi = t.run_wi.to(torch.int32)

    stream = torch.cuda.current_stream()
    split = {"push_s": 0.0, "compute_s": 0.0, "push_gpu_ms": 0.0, "compute_gpu_ms": 0.0}

    def step(measure=False):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        t0 = time.perf_counter()
        e0.record(stream)
        for c, t in zip(chars, traces):
            push_trace(c, t)
        e1.record(stream)
        t1 = time.perf_counter()
        out = compute_batch(chars, want_hist=False)
        e2.record(stream)
        t2 = time.perf_counter()
        if measure:
            e2.synchronize()
            split["push_s"] += t1 - t0
            split["compute_s"] += t2 - t1
            split["push_gpu_ms"] += e0.elapsed_time(e1)
            split["compute_gpu_ms"] += e1.elapsed_time(e2)
        return out
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    l0 = P.aiwc_kernel_launches()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        outs = step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.steps
    clocks = sampler.stop()
    launches = P.aiwc_kernel_launches() - l0
    # the same steps again, each split into its pushes and its batched compute
    # (wall clock and CUDA events on the stream), outside the timed region
    for _ in range(args.steps):
        step(measure=True)
    breakdown = {k: round((v * 1e3 if k.endswith("_s") else v) / args.steps, 3) for k, v in split.items()}
    breakdown = {k.replace("_s", "_ms"): v for k, v in breakdown.items()}
    for c in chars:
        c.close()
    return base_line(args, world, world * n_mem / dt, dt * 1e3, {
        "config": {"workload": "batched: 512 invocations, memory events log-uniform 2^12..2^24, footprints "
                               "log-uniform 2^8..2^22, patterns stream/stencil/gemm/zipf/uniform; one "
                               "aiwc_compute_batch (one CUDA graph) per step",
                   "memory_events_per_step": n_mem, "timing": "wall clock per step incl. pushes, synchronised",
                   "plans": "the library's automatic plan per invocation (sort plan up to 2^15 memory events, "
                            "else hash plan with a table of at least n slots)"},
        "clocks": clocks, "gpu_launches": launches, "gpu_launches_per_step": launches / args.steps,
        "step_breakdown_ms": breakdown,
        "result_check": {"footprint_sum": sum(o["footprint"] for o in outs)}})


def run_serving(args, P, torch, local, world, rank):
    import synth
    from paper_1805_04207_gb300.serving import Server
    jobs = synth.serving_jobs(args.jobs, rate_hz=200.0, seed=rank)
    # a device pool of 16-byte memory and 8-byte branch events the chunks slice
    pool_mem = synth.pattern_trace("zipf", 1 << 24, 1 << 22, device="cuda", seed=rank).mem
    pool_mem = torch.cat([pool_mem, synth.pattern_trace("stencil", 1 << 24, 1 << 22, device="cuda",
                                                        seed=rank, stream=1).mem])
    pool_br = synth.large_branch(1 << 24, device="cuda", seed=rank)
    P_total = pool_mem.shape[0]

    def chunks_of(job):
        off = 0
        for c in job["chunks"]:
            c = min(c, P_total)
            start = (off * 7919) % (P_total - c + 1)
            yield pool_mem[start:start + c]
            off += c
    srv = Server(device=local, max_jobs=32, workers=8, hbm_budget=120 << 30)
    lat, events = [], 0
    pending = list(jobs)
    running = {}
    sampler = ClockSampler(local)
    t0 = time.perf_counter()
    while pending or running:
        now = time.perf_counter() - t0
        while pending and pending[0]["arrival_s"] <= now:
            jb = pending[0]
            n_br = jb["n_mem"] // 4
            # device bytes a handle holds: about 19 B per memory event, 33 B per branch event, plus
            # fixed scratch (64 MB staging pair, table, work-item bitmap, arena)
            reserve = 24 * jb["n_mem"] + 40 * n_br + (256 << 20)
            # a streamed job's first chunk does not show its size; the caller
            # knows it and sizes the superblock table (a larger one needs no regrowth)
            slots = 1 << max(12, min(20, (jb["n_mem"] - 1).bit_length()))
            h = srv.open(reserve, n_opcodes=64, max_work_items=1 << 26, table_slots=slots)
            if h is None:
                break
            for ch in chunks_of(jb):
                h.push_mem(ch)
            left = n_br
            while left > 0:
                c = min(left, pool_br.shape[0])
                h.push_branch(pool_br[:c])
                left -= c
            h.finish()
            running[id(h)] = (jb, h)
            pending.pop(0)
            events += jb["n_mem"]
        for k, (jb, h) in list(running.items()):
            r = h.poll()
            if r is not None:
                lat.append(time.perf_counter() - t0 - jb["arrival_s"])
                del running[k]
    span = time.perf_counter() - t0
    clocks = sampler.stop()
    st = srv.stats()
    srv.close()
    lat.sort()
    p50 = lat[len(lat) // 2] if lat else None
    p99 = lat[min(len(lat) - 1, int(0.99 * len(lat)))] if lat else None
    return base_line(args, world, world * events / span, span * 1e3, {
        "steps": 1, "config": {"workload": f"serving: {args.jobs} jobs, Poisson 200/s, traces log-uniform "
                                           "16 MB..8 GB, chunks log-uniform 1..256 MB (device-resident pool), "
                                           "32 slots, 120 GiB budget",
                               "memory_events": events},
        "latency_s": {"p50": p50, "p99": p99, "max": lat[-1] if lat else None},
        "server": st, "clocks": clocks})


def run_precision(args, P, torch, local, world, rank):
    import synth
    from paper_1805_04207_gb300.api import push_trace
    s = args.scale
    tr = synth.precision(device="cuda", seed=rank, n_mem=1 << (30 - s), uniform_distinct=1 << (27 - s),
                         hot_distinct=1 << (20 - s), n_br=1 << (26 - s))
    tr.run_wi = tr.run_wi.to(torch.int32)
    res, times = {}, {}
    for prec in (0, 1):
        c = P.Characterizer(device=local, precision=prec, n_opcodes=tr.n_opcodes)
        for _ in range(max(3, args.warmup)):
            push_trace(c, tr)
            res[prec] = c.compute(want_hist=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            push_trace(c, tr)
            res[prec] = c.compute(want_hist=False)
        torch.cuda.synchronize()
        times[prec] = (time.perf_counter() - t0) / args.steps
        c.close()
    err = {f"entropy[{n}]": abs(res[1]["entropy"][n] - res[0]["entropy"][n]) for n in range(11)}
    err["albe"] = abs(res[1]["albe"] - res[0]["albe"])
    same_counts = all(res[1][k] == res[0][k] for k in ("footprint", "footprint_cover", "unique_reads",
                                                         "unique_writes", "branch_minsum", "branch_patterns"))
    return base_line(args, world, world * tr.n_mem / times[1], times[1] * 1e3, {
        "dtype": "u64+f32(compensated)",
        "config": {"workload": f"precision: 2^{30 - s} memory events, 75% uniform over 2^{27 - s} addresses + "
                               f"25% Zipf(1.2) over a 2^{20 - s} hot set; 2^{26 - s} branch events",
                   "timing": "wall clock per invocation incl. pushes, synchronised"},
        "fp32_vs_fp64_abs_error_bits": err, "max_abs_error_bits": max(err.values()), "bound_bits": 2.0 ** -22,
        "counts_identical": same_counts, "fp64_ms_per_step": round(times[0] * 1e3, 3)})


def run_partitioned(args, P, torch, local, world, rank):
    """An invocation held in host memory, reduced in 1 and in P partitions:
    time per invocation (routing and host-to-device copies included) and the
    device memory the handle holds."""
    import synth
    from paper_1805_04207_gb300.api import push_trace
    s = args.scale
    tr = synth.large(device="cpu", seed=rank, n_mem=1 << (26 - s), n_br=1 << (24 - s), n_wi=1 << (18 - s),
                     per_wi=1024, zipf_distinct=1 << (24 - s))
    tr.run_wi = tr.run_wi.to(torch.int32)
    for t in ("mem", "br", "ops", "run_wi", "run_off", "run_len"):
        setattr(tr, t, getattr(tr, t).contiguous().pin_memory())
    out, times, held = {}, {}, {}
    for parts in (1, args.partitions):
        c = P.Characterizer(device=local, n_opcodes=tr.n_opcodes, partitions=parts)
        for _ in range(max(3, args.warmup)):
            push_trace(c, tr)
            out[parts] = c.compute(want_hist=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            push_trace(c, tr)
            out[parts] = c.compute(want_hist=False)
        torch.cuda.synchronize()
        times[parts] = (time.perf_counter() - t0) / args.steps
        held[parts] = P.aiwc_device_bytes(c.h)
        c.close()
    a, b = out[1], out[args.partitions]
    same = all(a[k] == b[k] for k in a if not isinstance(a[k], (float, list))) and \
        max(abs(x - y) for x, y in zip(a["entropy"], b["entropy"])) < 1e-12
    return base_line(args, world, world * tr.n_mem / times[args.partitions], times[args.partitions] * 1e3, {
        "config": {"workload": f"partitioned: host-resident invocation of 2^{26 - s} memory, 2^{24 - s} branch, "
                               f"2^{28 - s} opcode events (large-invocation shapes) in {args.partitions} "
                               f"partitions", "timing": "wall clock per invocation incl. routing and copies"},
        "partitions": args.partitions, "device_bytes": held[args.partitions], "device_bytes_unpartitioned": held[1],
        "ms_per_step_unpartitioned": round(times[1] * 1e3, 3), "results_identical": same})


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload != "large":
        import torch
        import paper_1805_04207_gb300 as P
        torch.cuda.set_device(local)
        fn = {"batched": run_batched, "serving": run_serving, "precision": run_precision,
              "partitioned": run_partitioned}[args.workload]
        line = fn(args, P, torch, local, world, rank)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return

    import torch
    import paper_1805_04207_gb300 as P
    import synth
    from paper_1805_04207_gb300.api import push_trace

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    s = args.scale
    n_mem, n_br, n_wi = 1 << (28 - s), 1 << (26 - s), 1 << (20 - s)
    tr = synth.large(device="cuda", seed=rank, n_mem=n_mem, n_br=n_br, n_wi=n_wi, per_wi=1024,
                     zipf_distinct=1 << (26 - s))
    run_wi32 = tr.run_wi.to(torch.int32)
    n_ops = tr.n_ops
    in_bytes = 16 * n_mem + 8 * n_br + 2 * n_ops + (4 + 8 + 8) * tr.run_wi.numel()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    opts = options(args)
    c = P.Characterizer(device=local, stream=stream, n_opcodes=tr.n_opcodes, **opts)

    def step():
        c.push_mem(tr.mem)
        c.push_branch(tr.br)
        c.push_instr_runs(run_wi32, tr.run_off, tr.run_len, tr.ops)
        return c.compute(want_hist=False)

    for _ in range(max(3, args.warmup)):
        out = step()
    # timed region: device-resident inputs, CUDA events on the handle's stream
    c.set_stage_timing(True)
    stage_tot = {}
    barrier()
    sampler = ClockSampler(local)
    l0 = P.aiwc_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        out = step()
        for k, v in c.stage_times().items():
            stage_tot[k] = stage_tot.get(k, 0.0) + v
    ev1.record(stream)
    barrier()
    clocks = sampler.stop()
    launches = P.aiwc_kernel_launches() - l0
    c.set_stage_timing(False)
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms, dist, "cuda")
    value = replica_throughput(n_mem * args.steps, world, ms_max / 1e3)

    # roofline of the dominant stage, plus the whole step
    hbm, peak_kind = peaks()
    per_step = {k: v / args.steps for k, v in stage_tot.items()}
    D = out["footprint"]
    Bp = out["branch_patterns"]
    # with byte-granular addresses the byte count pass and the ingest each read
    # the 16-byte events once (the one-byte accesses are formed on chip)
    byte_mode = bool(opts.get("byte_addresses"))
    n_acc = out["total_reads"] + out["total_writes"] if byte_mode else n_mem
    alg = {"mem_ingest": ALG_BYTES["mem_event"] * n_mem,
           "branch_ingest": ALG_BYTES["branch_event"] * n_br,
           "mem_expand": ALG_BYTES["mem_event"] * n_mem,
           "instr_runs": ALG_BYTES["opcode"] * n_ops,
           "mem_sort": 16 * n_acc, "mem_scatter": 0, "mem_levels": ALG_BYTES["distinct_key"] * D,
           "branch_sort": 16 * n_br, "windows": ALG_BYTES["pattern"] * Bp, "pattern_sort": 16 * Bp,
           "pattern_runs": 0, "run_sort": 16 * tr.run_wi.numel(),
           "run_combine": 0, "finalize": 0}
    dom = max(per_step, key=per_step.get)
    dom_ms = per_step[dom]
    achieved = alg.get(dom, 0) / (dom_ms / 1e3) / 1e9 if dom_ms > 0 else 0.0
    step_alg = (ALG_BYTES["mem_event"] * n_mem + ALG_BYTES["branch_event"] * n_br + ALG_BYTES["opcode"] * n_ops +
                ALG_BYTES["distinct_key"] * D + ALG_BYTES["pattern"] * Bp)
    step_ach = step_alg / (ms_max / args.steps / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4),
            # the committed counters describe the event ingest, not the byte ingest
            "traffic": None if byte_mode else traffic_for(dom), "peak_kind": peak_kind,
            "alg_bytes_per_launch": alg.get(dom, 0), "ms_per_launch": round(dom_ms, 4)}

    # end to end through the public API from pinned host buffers
    e2e = None
    if not args.no_e2e:
        hmem = tr.mem.cpu().pin_memory()
        hbr = tr.br.cpu().pin_memory()
        hops = tr.ops.cpu().pin_memory()
        hwi, hoff, hlen = run_wi32.cpu().pin_memory(), tr.run_off.cpu().pin_memory(), tr.run_len.cpu().pin_memory()

        def hstep():
            c.push_mem(hmem)
            c.push_branch(hbr)
            c.push_instr_runs(hwi, hoff, hlen, hops)
            return c.compute(want_hist=True)
        hstep()
        barrier()
        t0 = time.perf_counter()
        ek = max(1, min(args.steps, 3))
        for _ in range(ek):
            hstep()
        barrier()
        e_s = max_over_ranks((time.perf_counter() - t0) / ek, dist, "cuda")
        h2d = 16 * n_mem + 8 * n_br + 2 * n_ops + (4 + 8 + 8) * tr.run_wi.numel()
        d2h = 8 * 11 + 8 * 40 + 8 * tr.n_opcodes
        e2e = {"value": replica_throughput(n_mem, world, e_s), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": round(e_s * 1e3, 3), "steps": ek}
        del hmem, hbr, hops

    base = base_all = None
    if rank == 0 and not args.no_cpu_baseline:
        base, _ = cpu_baseline(s, opts)
        try:
            base_all = cpu_baseline_all_cores(s + 3, opts)
        except Exception as e:  # a reported baseline only: never lose the bench line to it
            base_all = {"unavailable": f"{type(e).__name__}: {e}"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": round(ms_max / args.steps, 4),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64+f64",
                "data": "synthetic", "impl": "ours",
                "config": {"workload": workload_name(args), "seed": "rank",
                           "inputs": inputs_note(in_bytes),
                           "parallelism": f"replicas x{world}", "scale_shift": s, **opts},
                "roofline": roof,
                "roofline_step": {"bound": "hbm", "achieved": round(step_ach, 1), "peak": hbm, "unit": "GB/s",
                                  "frac": round(step_ach / hbm, 4), "alg_bytes_per_step": step_alg},
                "stage_ms_per_step": {k: round(v, 4) for k, v in per_step.items()},
                "e2e": e2e, "cpu_baseline": base, "cpu_baseline_all_cores": base_all,
                "clocks": clocks, "gpu_launches": launches,
                "gpu_launches_per_step": launches / args.steps,
                "result_check": {"footprint": D, "entropy0": out["entropy"][0], "albe": out["albe"],
                                 "itb_median": out["itb_median"], "work_items": out["work_items"]}}
        print(json.dumps(line), flush=True)
    c.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
