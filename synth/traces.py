"""Counter-based synthetic AIWC traces (see the package docstring for layouts).

The workloads stand in for the Extended OpenDwarfs kernels run under Oclgrind
that the paper characterises (Sec. VI); neither the suite nor the simulator is
used. Shapes follow the kernels the paper discusses: strided and gathered
float32 accesses, a 7-point stencil, a 16x16-tiled SGEMM, Zipf-distributed
gathers, loop back-edges and data-dependent branches, and instruction streams
with periodic barriers (Sec. VI reports one barrier per 25 instructions for
needle; the tiny workload uses 1 per 500, the large one 1 per 100).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

_M64 = (1 << 64) - 1


def _s64(v: int) -> int:
    """Reinterpret an unsigned 64-bit Python int as a signed int64 value."""
    v &= _M64
    return v - (1 << 64) if v >> 63 else v


_GOLD = _s64(0x9E3779B97F4A7C15)
_M1 = _s64(0xBF58476D1CE4E5B9)
_M2 = _s64(0x94D049BB133111EB)

BARRIER_I16 = -1  # 0xFFFF stored as int16


def _srl(x: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of an int64 tensor holding unsigned 64-bit words."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def mix64(x: torch.Tensor) -> torch.Tensor:
    """SplitMix64 output function on int64 tensors (wrapping arithmetic)."""
    x = x ^ _srl(x, 30)
    x = x * _M1
    x = x ^ _srl(x, 27)
    x = x * _M2
    return x ^ _srl(x, 31)


def _mix64_int(v: int) -> int:
    v &= _M64
    v ^= v >> 30
    v = (v * 0xBF58476D1CE4E5B9) & _M64
    v ^= v >> 27
    v = (v * 0x94D049BB133111EB) & _M64
    return v ^ (v >> 31)


def hash3(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """64-bit hash of (seed, stream, idx); idx is an int64 tensor of counters."""
    key = _mix64_int(_mix64_int(seed * 0x9E3779B97F4A7C15 + 0x632BE59BD9B4E019)
                     + stream * 0x9E3779B97F4A7C15)
    return mix64(idx * _GOLD + _s64(key))


def u01(h: torch.Tensor) -> torch.Tensor:
    """Uniform double in [0, 1) from the top 53 bits of a hash word."""
    return _srl(h, 11).to(torch.float64) * (1.0 / 9007199254740992.0)


def _below(h: torch.Tensor, m) -> torch.Tensor:
    """Integer in [0, m) from a hash word (m an int or an int64 tensor)."""
    return _srl(h, 1) % m


def _perm(x: torch.Tensor, bits: int) -> torch.Tensor:
    """A bijection of [0, 2**bits): odd multiply, xorshift, odd multiply."""
    if bits == 0:
        return torch.zeros_like(x)
    mask = (1 << bits) - 1
    y = (x * 0x2545F491) & mask
    y = y ^ (y >> max(1, (bits + 1) // 2))
    return (y * 0x5851F42D) & mask


_ZIPF_CDF: dict = {}


def zipf_rank(u: torch.Tensor, n: int, s: float) -> torch.Tensor:
    """Rank in [0, n) with P(rank = k) proportional to (k + 1)**-s.

    Inverts the discrete CDF by binary search. The CDF table is built once on
    the CPU in float64 and shared by every device, so ranks are identical on
    the CPU and on a GPU for the same uniforms.
    """
    key = (n, float(s), str(u.device))
    cdf = _ZIPF_CDF.get(key)
    if cdf is None:
        host = _ZIPF_CDF.get((n, float(s), "cpu"))
        if host is None:
            w = torch.arange(1, n + 1, dtype=torch.float64).pow_(-float(s))
            host = torch.cumsum(w, 0)
            host /= host[-1].clone()
            _ZIPF_CDF[(n, float(s), "cpu")] = host
        cdf = host.to(u.device)
        _ZIPF_CDF[key] = cdf
    return torch.searchsorted(cdf, u, right=True).clamp_(max=n - 1)


def pack_mem(addr, wi, size, store, space) -> torch.Tensor:
    """Pack memory events into the 16-byte layout, as an (n, 2) int64 tensor."""
    addr = torch.as_tensor(addr, dtype=torch.int64)
    n = addr.shape[0]
    out = torch.empty((n, 2), dtype=torch.int64, device=addr.device)
    out[:, 0] = addr
    flags = (torch.as_tensor(store, dtype=torch.int64, device=addr.device) & 1) | \
        ((torch.as_tensor(space, dtype=torch.int64, device=addr.device) & 3) << 1)
    out[:, 1] = (torch.as_tensor(wi, dtype=torch.int64, device=addr.device) & 0xFFFFFFFF) | \
        ((torch.as_tensor(size, dtype=torch.int64, device=addr.device) & 0xFF) << 32) | (flags << 40)
    return out


def pack_branch(site, wi, taken) -> torch.Tensor:
    """Pack branch events into the 8-byte layout, as an (n,) int64 tensor."""
    site = torch.as_tensor(site, dtype=torch.int64)
    dev = site.device
    hi = (torch.as_tensor(wi, dtype=torch.int64, device=dev) & 0x7FFFFFFF) | \
        ((torch.as_tensor(taken, dtype=torch.int64, device=dev) & 1) << 31)
    return (site & 0xFFFFFFFF) | (hi << 32)


@dataclass
class Trace:
    """One kernel invocation's three event streams plus the run table."""
    name: str
    mem: torch.Tensor | None = None      # (n, 2) int64, 16-byte memory events
    br: torch.Tensor | None = None       # (n,) int64, 8-byte branch events
    ops: torch.Tensor | None = None      # (I,) int16 opcodes, -1 = barrier
    run_wi: torch.Tensor | None = None   # (R,) int64 work-item of each run
    run_off: torch.Tensor | None = None  # (R,) int64 offset of each run in ops
    run_len: torch.Tensor | None = None  # (R,) int64 length of each run
    n_opcodes: int = 65535
    meta: dict = field(default_factory=dict)
    widths: torch.Tensor | None = None   # (I',) int16 result width of each counted instruction

    def to(self, device) -> "Trace":
        def mv(t):
            return None if t is None else t.to(device)
        return Trace(self.name, mv(self.mem), mv(self.br), mv(self.ops), mv(self.run_wi),
                     mv(self.run_off), mv(self.run_len), self.n_opcodes, dict(self.meta), mv(self.widths))

    @property
    def n_mem(self) -> int:
        return 0 if self.mem is None else int(self.mem.shape[0])

    @property
    def n_br(self) -> int:
        return 0 if self.br is None else int(self.br.shape[0])

    @property
    def n_ops(self) -> int:
        return 0 if self.ops is None else int(self.ops.shape[0])

    def nbytes(self) -> int:
        nw = 0 if self.widths is None else int(self.widths.shape[0])
        return 16 * self.n_mem + 8 * self.n_br + 2 * self.n_ops + 2 * nw


def _blocks(n: int, block: int = 1 << 24):
    for lo in range(0, n, block):
        yield lo, min(n, lo + block)


# --------------------------------------------------------------------------
# Tiny workload: 256 work-items; 65,536 memory, 8,192 branch, 200,000
# instruction events.
# --------------------------------------------------------------------------

def tiny(device="cpu", seed: int = 0) -> Trace:
    dev = torch.device(device)
    W = 256
    n_mem = 65536
    i = torch.arange(n_mem, dtype=torch.int64, device=dev)
    gather = (i % 4) == 3
    # stride-4 float32 reads over a 16 KiB __local array (4096 elements)
    s_idx = (4 * i + (i >> 10)) % 4096
    s_addr = 0x1000 + 4 * s_idx
    # Zipf(1.1) gathers over 4096 float32 elements of a __global array
    rank = zipf_rank(u01(hash3(seed, 0, i)), 4096, 1.1)
    g_addr = (1 << 40) + 4 * _perm(rank, 12)
    addr = torch.where(gather, g_addr, s_addr)
    space = torch.where(gather, torch.zeros_like(i), torch.ones_like(i))
    store = (u01(hash3(seed, 1, i)) < 0.3).to(torch.int64)
    mem = pack_mem(addr, i % W, torch.full_like(i, 4), store, space)

    # 8,192 branch events: pushed as (k, w, s) with 2 events per (work-item,
    # site); site 15 is a fair coin, sites 0..14 are loop back-edges taken 31
    # of every 32 times in their per-site (work-item, program order) sequence.
    e = torch.arange(2 * W * 16, dtype=torch.int64, device=dev)
    s = e % 16
    w = (e // 16) % W
    k = e // (16 * W)
    j = 2 * w + k
    loop_taken = (j % 32) != 31
    coin = u01(hash3(seed, 2, e)) < 0.5
    taken = torch.where(s == 15, coin, loop_taken).to(torch.int64)
    br = pack_branch(s, w, taken)

    # 200,000 instructions over 64 opcodes in one run per work-item; a
    # barrier marker after the 500th instruction of each work-item.
    lens = torch.tensor([782 if ww < 64 else 781 for ww in range(W)], dtype=torch.int64)
    run_len = lens + 1
    run_off = torch.cumsum(run_len, 0) - run_len
    total = int(run_len.sum())
    g = torch.arange(total, dtype=torch.int64)
    wi_of = torch.repeat_interleave(torch.arange(W, dtype=torch.int64), run_len)
    pos = g - run_off[wi_of]
    ops = (_below(hash3(seed, 3, g), 64)).to(torch.int16)
    ops[pos == 500] = BARRIER_I16
    # result widths of the counted instructions: 1, 2, 4, 8 or 16 data items
    n_counted = int((pos != 500).sum())
    widths = (1 << _below(hash3(seed, 4, torch.arange(n_counted, dtype=torch.int64)), 5)).to(torch.int16)
    return Trace("tiny", mem, br, ops.to(dev), torch.arange(W, dtype=torch.int64, device=dev),
                 run_off.to(dev), run_len.to(dev), n_opcodes=64,
                 meta={"seed": seed, "work_items": W}, widths=widths.to(dev))


# --------------------------------------------------------------------------
# Large workload: 7-point stencil + tiled SGEMM + Zipf gathers; loop and
# Bernoulli branches over 4,096 sites; 256-opcode instruction stream.
# --------------------------------------------------------------------------

_BUF_IN, _BUF_OUT, _BUF_A, _BUF_B, _BUF_C, _BUF_Z = (b << 40 for b in range(1, 7))


def _stencil_events(e: torch.Tensor):
    """7 reads + 1 write per point of a 256^3 float32 grid, point-major."""
    p = e // 8
    r = e % 8
    x = p % 256
    y = (p // 256) % 256
    z = (p // 65536) % 256
    dx = torch.where(r == 1, -1, torch.where(r == 2, 1, 0))
    dy = torch.where(r == 3, -1, torch.where(r == 4, 1, 0))
    dz = torch.where(r == 5, -1, torch.where(r == 6, 1, 0))
    idx = (((z + dz) % 256) * 256 + (y + dy) % 256) * 256 + (x + dx) % 256
    write = r == 7
    addr = torch.where(write, _BUF_OUT + 4 * (p % (1 << 24)), _BUF_IN + 4 * idx)
    return addr, p, write.to(torch.int64)


def _gemm_events(e: torch.Tensor, n: int = 2048):
    """First accesses of a 16x16-tiled SGEMM C = A B (n x n), work-group order."""
    tiles = n // 16
    per_wg = tiles * 512 + 256
    wg = e // per_wg
    rr = e % per_wg
    bi = (wg // tiles) % tiles
    bj = wg % tiles
    is_c = rr >= tiles * 512
    kt = rr // 512
    q = rr % 512
    t = torch.where(is_c, rr - tiles * 512, q % 256)
    ti = t // 16
    tj = t % 16
    is_b = (q >= 256) & ~is_c
    a_addr = _BUF_A + 4 * ((bi * 16 + ti) * n + kt * 16 + tj)
    b_addr = _BUF_B + 4 * ((kt * 16 + ti) * n + bj * 16 + tj)
    c_addr = _BUF_C + 4 * ((bi * 16 + ti) * n + bj * 16 + tj)
    addr = torch.where(is_c, c_addr, torch.where(is_b, b_addr, a_addr))
    wi = (bi * 16 + ti) * n + bj * 16 + tj
    return addr, wi, is_c.to(torch.int64)


def _zipf_events(seed: int, e: torch.Tensor, n_distinct: int, s: float, base: int, stream: int,
                 wi_div: int = 64, p_store: float = 0.1):
    bits = int(math.log2(n_distinct))
    assert 1 << bits == n_distinct
    rank = zipf_rank(u01(hash3(seed, stream, e)), n_distinct, s)
    addr = base + 8 * _perm(rank, bits)
    store = (u01(hash3(seed, stream + 1, e)) < p_store).to(torch.int64)
    return addr, e // wi_div, store


def large_mem(n_mem: int, device="cpu", seed: int = 0, zipf_distinct: int = 1 << 26) -> torch.Tensor:
    """n_mem events: half stencil, a quarter SGEMM, a quarter Zipf(1.05) gathers."""
    dev = torch.device(device)
    n_st = n_mem // 2
    n_gm = n_mem // 4
    out = torch.empty((n_mem, 2), dtype=torch.int64, device=dev)
    for lo, hi in _blocks(n_mem):
        e = torch.arange(lo, hi, dtype=torch.int64, device=dev)
        st_addr, st_wi, st_w = _stencil_events(e)
        g = e - n_st
        gm_addr, gm_wi, gm_w = _gemm_events(g.clamp(min=0))
        z = e - n_st - n_gm
        zp_addr, zp_wi, zp_w = _zipf_events(seed, z.clamp(min=0), zipf_distinct, 1.05, _BUF_Z, 10)
        in_st = e < n_st
        in_gm = (e >= n_st) & (e < n_st + n_gm)
        addr = torch.where(in_st, st_addr, torch.where(in_gm, gm_addr, zp_addr))
        wi = torch.where(in_st, st_wi, torch.where(in_gm, gm_wi, zp_wi))
        st = torch.where(in_st, st_w, torch.where(in_gm, gm_w, zp_w))
        out[lo:hi] = pack_mem(addr, wi, 4 + 4 * (~(in_st | in_gm)).to(torch.int64), st, torch.zeros_like(e))
    return out


def large_branch(n_br: int, device="cpu", seed: int = 0, n_sites: int = 4096, per_wi: int = 1024) -> torch.Tensor:
    """Branch events in blocks of 16 per (work-item, site); 70% loop sites."""
    dev = torch.device(device)
    out = torch.empty((n_br,), dtype=torch.int64, device=dev)
    n_loop = (7 * n_sites) // 10
    for lo, hi in _blocks(n_br):
        i = torch.arange(lo, hi, dtype=torch.int64, device=dev)
        w = i // per_wi
        k = i % per_wi
        site = _below(hash3(seed, 20, w * per_wi + k // 16), n_sites)
        trip = 4 + _below(hash3(seed, 21, site), 61)
        loop_taken = (k % trip) != (trip - 1)
        p = u01(hash3(seed, 22, site))
        coin = u01(hash3(seed, 23, i)) < p
        taken = torch.where(site < n_loop, loop_taken, coin).to(torch.int64)
        out[lo:hi] = pack_branch(site, w, taken)
    return out


def large_instr(n_wi: int, per_wi: int = 1024, n_op_ids: int = 256, barrier_every: int = 100,
                device="cpu", seed: int = 0):
    """n_wi runs of per_wi slots; a barrier after every barrier_every instructions."""
    dev = torch.device(device)
    total = n_wi * per_wi
    ops = torch.empty((total,), dtype=torch.int16, device=dev)
    for lo, hi in _blocks(total):
        g = torch.arange(lo, hi, dtype=torch.int64, device=dev)
        op = _below(hash3(seed, 30, g), n_op_ids)
        is_bar = (g % per_wi) % (barrier_every + 1) == barrier_every
        ops[lo:hi] = torch.where(is_bar, torch.full_like(op, BARRIER_I16), op).to(torch.int16)
    run_wi = torch.arange(n_wi, dtype=torch.int64, device=dev)
    run_off = run_wi * per_wi
    run_len = torch.full((n_wi,), per_wi, dtype=torch.int64, device=dev)
    return ops, run_wi, run_off, run_len


def large(device="cpu", seed: int = 0, n_mem: int = 1 << 28, n_br: int = 1 << 26,
          n_wi: int = 1 << 20, per_wi: int = 1024, zipf_distinct: int = 1 << 26) -> Trace:
    """The large single invocation (defaults: 2^28 / 2^26 / 2^30 events).

    Smaller arguments give the same shapes at sizes the oracle finishes in
    seconds (the parity tests use ragged ones).
    """
    mem = large_mem(n_mem, device, seed, zipf_distinct)
    br = large_branch(n_br, device, seed)
    ops, rwi, roff, rlen = large_instr(n_wi, per_wi, device=device, seed=seed)
    return Trace("large", mem, br, ops, rwi, roff, rlen, n_opcodes=256,
                 meta={"seed": seed, "n_mem": n_mem, "n_br": n_br, "n_wi": n_wi, "per_wi": per_wi})


# --------------------------------------------------------------------------
# Precision workload: near-uniform accesses over 2^27 addresses plus a
# 2^20-address Zipf(1.2) hot set.
# --------------------------------------------------------------------------

def precision(device="cpu", seed: int = 0, n_mem: int = 1 << 30, uniform_distinct: int = 1 << 27,
              hot_distinct: int = 1 << 20, n_br: int = 1 << 26, n_wi: int = 1 << 12) -> Trace:
    dev = torch.device(device)
    mem = torch.empty((n_mem, 2), dtype=torch.int64, device=dev)
    n_uni = (3 * n_mem) // 4
    for lo, hi in _blocks(n_mem):
        e = torch.arange(lo, hi, dtype=torch.int64, device=dev)
        u_addr = (7 << 40) + 8 * _below(hash3(seed, 40, e), uniform_distinct)
        z_addr, _, _ = _zipf_events(seed, e, hot_distinct, 1.2, 8 << 40, 41)
        is_u = e < n_uni
        addr = torch.where(is_u, u_addr, z_addr)
        store = (u01(hash3(seed, 43, e)) < 0.1).to(torch.int64)
        mem[lo:hi] = pack_mem(addr, e // 256, torch.full_like(e, 8), store, torch.zeros_like(e))
    br = large_branch(n_br, device, seed)
    ops, rwi, roff, rlen = large_instr(n_wi, device=device, seed=seed)
    return Trace("precision", mem, br, ops, rwi, roff, rlen, n_opcodes=256,
                 meta={"seed": seed, "n_mem": n_mem})


# --------------------------------------------------------------------------
# Batched workload: many invocations of uneven length and footprint.
# --------------------------------------------------------------------------

PATTERNS = ("stream", "stencil", "gemm", "zipf", "uniform")


def pattern_trace(kind: str, count: int, footprint: int, device="cpu", seed: int = 0,
                  stream: int = 0) -> Trace:
    """One invocation with `count` memory events drawn from `footprint` addresses.

    Branch events = count/4 and instruction events = 4*count, shaped like the
    tiny workload (16 sites; a barrier every 500 instructions).
    """
    dev = torch.device(device)
    F = max(1, min(footprint, count))
    e = torch.arange(count, dtype=torch.int64, device=dev)
    h = hash3(seed, 100 + stream, e)
    base = (1 + (stream % 1000)) << 32
    if kind == "stream":
        idx = e % F
        store = (e % 8 == 7)
    elif kind == "stencil":
        p = e // 4
        r = e % 4
        idx = torch.where(r == 0, p - 1, torch.where(r == 2, p + 1, p)) % F
        store = r == 3
    elif kind == "gemm":
        n = max(16, (int(math.isqrt(F)) // 16) * 16)
        a, _, c = _gemm_events(e, n)
        idx = ((a - _BUF_A) // 4) % F
        store = c.bool()
    elif kind == "zipf":
        Fp = 1 << max(0, (F - 1).bit_length())
        idx = zipf_rank(u01(h), Fp, 1.1)
        idx = _perm(idx, Fp.bit_length() - 1) % F
        store = u01(hash3(seed, 200 + stream, e)) < 0.1
    elif kind == "uniform":
        idx = _below(h, F)
        store = u01(hash3(seed, 200 + stream, e)) < 0.2
    else:
        raise ValueError(kind)
    W = max(1, count // 256)
    mem = pack_mem(base + 4 * idx, e % W, torch.full_like(e, 4), store.to(torch.int64),
                   torch.zeros_like(e))
    nb = max(0, count // 4)
    b = torch.arange(nb, dtype=torch.int64, device=dev)
    s = b % 16
    wb = (b // 16) % W
    j = b // 16
    taken = torch.where(s == 15, u01(hash3(seed, 300 + stream, b)) < 0.5, (j % 32) != 31)
    br = pack_branch(s, wb, taken.to(torch.int64))
    n_ops = 4 * count
    per = max(1, n_ops // W)
    lens = torch.full((W,), per, dtype=torch.int64)
    lens[-1] += n_ops - per * W
    run_off = torch.cumsum(lens, 0) - lens
    g = torch.arange(n_ops, dtype=torch.int64, device=dev)
    op = _below(hash3(seed, 400 + stream, g), 64)
    wi_of = torch.repeat_interleave(torch.arange(W, dtype=torch.int64, device=dev), lens.to(dev))
    pos = g - run_off.to(dev)[wi_of]
    op = torch.where(pos % 501 == 500, torch.full_like(op, BARRIER_I16), op).to(torch.int16)
    return Trace(f"{kind}:{count}:{F}", mem, br, op, torch.arange(W, dtype=torch.int64, device=dev),
                 run_off.to(dev), lens.to(dev), n_opcodes=64,
                 meta={"kind": kind, "count": count, "footprint": F})


def batched(n_traces: int = 512, device="cpu", seed: int = 0, lo_log2: int = 12, hi_log2: int = 24,
            f_lo_log2: int = 8, f_hi_log2: int = 22) -> list[Trace]:
    """Invocation traces with log-uniform event counts and footprints."""
    t = torch.arange(n_traces, dtype=torch.int64)
    uc = u01(hash3(seed, 500, t))
    uf = u01(hash3(seed, 501, t))
    uk = _below(hash3(seed, 502, t), len(PATTERNS))
    out = []
    for k in range(n_traces):
        count = int(round(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * float(uc[k]))))
        F = int(round(2.0 ** (f_lo_log2 + (f_hi_log2 - f_lo_log2) * float(uf[k]))))
        out.append(pattern_trace(PATTERNS[int(uk[k])], count, min(F, count), device, seed, k))
    return out


def serving_jobs(n_jobs: int, rate_hz: float = 200.0, seed: int = 0, lo_bytes: float = 16e6,
                 hi_bytes: float = 8e9, chunk_lo: float = 1e6, chunk_hi: float = 256e6):
    """Poisson job arrivals with log-uniform sizes and chunkings.

    Returns a list of dicts: arrival time (s), total memory events, pattern,
    footprint and the chunk sizes (in memory events) the job streams in.
    """
    t = torch.arange(n_jobs, dtype=torch.int64)
    gaps = -torch.log1p(-u01(hash3(seed, 600, t))) / rate_hz
    arrivals = torch.cumsum(gaps, 0)
    jobs = []
    for j in range(n_jobs):
        hj = torch.tensor([j], dtype=torch.int64)
        ub = float(u01(hash3(seed, 601, hj)))
        nbytes = math.exp(math.log(lo_bytes) + (math.log(hi_bytes) - math.log(lo_bytes)) * ub)
        n_mem = max(1 << 12, int(nbytes * 0.75) // 16)
        kind = PATTERNS[int(_below(hash3(seed, 602, hj), len(PATTERNS)))]
        uf = float(u01(hash3(seed, 603, hj)))
        F = max(256, min(n_mem, int(2 ** (8 + 14 * uf))))
        chunks = []
        left = n_mem
        c = 0
        while left > 0:
            uc = float(u01(hash3(seed, 604 + j, torch.tensor([c], dtype=torch.int64))))
            cb = math.exp(math.log(chunk_lo) + (math.log(chunk_hi) - math.log(chunk_lo)) * uc)
            ce = max(1, min(left, int(cb) // 16))
            chunks.append(ce)
            left -= ce
            c += 1
        jobs.append({"job": j, "arrival_s": float(arrivals[j]), "n_mem": n_mem, "kind": kind,
                     "footprint": F, "chunks": chunks})
    return jobs
