"""GB300-native reduction of OpenCL kernel event traces to the AIWC metrics.

Thin ctypes binding over ``libaiwc.so`` (C ABI in ``include/aiwc.h``). Every
step of the reduction runs in the library's CUDA kernels; this module only
marshals arguments. PyTorch is used for device memory and streams: tensors
are passed by ``data_ptr()`` and streams by ``torch.cuda.Stream.cuda_stream``.

Importing the package loads the library and raises if it has not been built
(``python -m paper_1805_04207_gb300._build``); there is no other code path.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

AIWC_OK, AIWC_EINVAL, AIWC_ENOMEM, AIWC_ECUDA, AIWC_ESTATE, AIWC_ETIMEOUT, AIWC_EAGAIN = range(7)
STATUS_NAMES = {0: "AIWC_OK", 1: "AIWC_EINVAL", 2: "AIWC_ENOMEM", 3: "AIWC_ECUDA", 4: "AIWC_ESTATE",
                5: "AIWC_ETIMEOUT", 6: "AIWC_EAGAIN"}
AIWC_BARRIER = 0xFFFF
MAX_SKIP = 10


class aiwc_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("cuda_stream", ctypes.c_void_p), ("history_len", ctypes.c_uint32),
                ("cover_num", ctypes.c_uint32), ("cover_den", ctypes.c_uint32), ("n_opcodes", ctypes.c_uint32),
                ("space_mask", ctypes.c_uint32), ("precision", ctypes.c_uint32), ("plan", ctypes.c_uint32),
                ("max_work_items", ctypes.c_uint64), ("hbm_budget", ctypes.c_uint64),
                ("table_slots", ctypes.c_uint64), ("partitions", ctypes.c_uint32),
                ("byte_addresses", ctypes.c_uint32), ("history_scope", ctypes.c_uint32),
                ("defer_pushes", ctypes.c_uint32)]


class aiwc_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("max_jobs", ctypes.c_uint32), ("workers", ctypes.c_uint32),
                ("hbm_budget", ctypes.c_uint64)]


_U64 = ctypes.c_uint64
_F64 = ctypes.c_double
METRIC_FIELDS = [
    ("total_instructions", _U64), ("unique_opcodes", _U64), ("opcode_cover", _U64),
    ("work_items", _U64), ("barriers", _U64),
    ("itb_count", _U64), ("itb_min", _U64), ("itb_max", _U64), ("itb_median_lo", _U64), ("itb_median_hi", _U64),
    ("itb_median", _F64),
    ("ipt_count", _U64), ("ipt_min", _U64), ("ipt_max", _U64), ("ipt_median_lo", _U64), ("ipt_median_hi", _U64),
    ("ipt_median", _F64),
    ("total_reads", _U64), ("total_writes", _U64), ("footprint", _U64), ("footprint_cover", _U64),
    ("unique_reads", _U64), ("unique_writes", _U64),
    ("entropy", _F64 * (MAX_SKIP + 1)),
    ("branch_events", _U64), ("branch_sites", _U64), ("branch_cover", _U64), ("branch_patterns", _U64),
    ("branch_minsum", _U64), ("albe", _F64), ("yokota", _F64),
    ("unique_rw_ratio", _F64), ("reread_ratio", _F64), ("rewrite_ratio", _F64),
    ("simd_count", _U64), ("simd_max", _U64), ("simd_sum", _U64), ("simd_sumsq", _U64),
    ("simd_mean", _F64), ("simd_sd", _F64),
    ("granularity", _F64), ("barriers_per_instruction", _F64), ("instructions_per_operand", _F64),
    ("load_imbalance", _F64),
    ("opcode_hist", ctypes.POINTER(ctypes.c_uint64)),
]
AGG_SUM = 0
AGG_MEDIAN = 1


class aiwc_metrics(ctypes.Structure):
    _fields_ = METRIC_FIELDS


# Every entry point declared in include/aiwc.h: name -> (restype, argtypes).
_VP = ctypes.c_void_p
_SZ = ctypes.c_size_t
_ST = ctypes.c_int
SIGNATURES = {
    "aiwc_config_default": (None, [ctypes.POINTER(aiwc_config)]),
    "aiwc_create": (_ST, [ctypes.POINTER(aiwc_config), ctypes.POINTER(_VP)]),
    "aiwc_push_mem": (_ST, [_VP, _VP, _SZ, ctypes.c_int]),
    "aiwc_push_branch": (_ST, [_VP, _VP, _SZ, ctypes.c_int]),
    "aiwc_push_instr": (_ST, [_VP, ctypes.c_uint32, _VP, _SZ, ctypes.c_int]),
    "aiwc_push_widths": (_ST, [_VP, _VP, _SZ, ctypes.c_int]),
    "aiwc_aggregate": (_ST, [ctypes.POINTER(aiwc_metrics), _SZ, ctypes.c_int, ctypes.POINTER(aiwc_metrics)]),
    "aiwc_push_instr_runs": (_ST, [_VP, _VP, _VP, _VP, _SZ, _VP, _SZ, ctypes.c_int]),
    "aiwc_compute": (_ST, [_VP, ctypes.POINTER(aiwc_metrics)]),
    "aiwc_compute_batch": (_ST, [ctypes.POINTER(_VP), _SZ, ctypes.POINTER(aiwc_metrics)]),
    "aiwc_destroy": (_ST, [_VP]),
    "aiwc_last_error": (ctypes.c_char_p, [_VP]),
    "aiwc_device_bytes": (ctypes.c_uint64, [_VP]),
    "aiwc_kernel_launches": (ctypes.c_uint64, []),
    "aiwc_set_stage_timing": (_ST, [_VP, ctypes.c_int]),
    "aiwc_stage_times": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_char_p),
                                        ctypes.c_int]),
    "aiwc_shard_route_mem": (_ST, [ctypes.c_uint32, ctypes.c_int, _VP, _SZ, _VP, _SZ, _VP, ctypes.POINTER(_SZ)]),
    "aiwc_shard_route_branch": (_ST, [ctypes.c_uint32, _VP, _SZ, _VP, _VP]),
    "aiwc_shard_route_runs": (_ST, [ctypes.c_uint32, _VP, _VP, _VP, _SZ, _VP, _SZ, _VP, _VP, _VP, _VP, _VP, _VP]),
    "aiwc_shard_export": (_ST, [_VP, _VP, _SZ, ctypes.POINTER(_SZ)]),
    "aiwc_shard_merge": (_ST, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_SZ), _SZ, ctypes.POINTER(aiwc_metrics)]),
    "aiwc_mem_metrics_noalloc": (_ST, [ctypes.c_int, _VP, _VP, _SZ, ctypes.c_uint32, ctypes.POINTER(aiwc_metrics)]),
    "aiwc_server_config_default": (None, [ctypes.POINTER(aiwc_server_config)]),
    "aiwc_server_create": (_ST, [ctypes.POINTER(aiwc_server_config), ctypes.POINTER(_VP)]),
    "aiwc_job_open": (_ST, [_VP, ctypes.POINTER(aiwc_config), ctypes.c_uint64, ctypes.POINTER(_VP)]),
    "aiwc_job_push_mem": (_ST, [_VP, _VP, _SZ, ctypes.c_int]),
    "aiwc_job_push_branch": (_ST, [_VP, _VP, _SZ, ctypes.c_int]),
    "aiwc_job_push_widths": (_ST, [_VP, _VP, _SZ, ctypes.c_int]),
    "aiwc_job_push_instr_runs": (_ST, [_VP, _VP, _VP, _VP, _SZ, _VP, _SZ, ctypes.c_int]),
    "aiwc_job_finish": (_ST, [_VP]),
    "aiwc_job_poll": (_ST, [_VP, ctypes.POINTER(aiwc_metrics)]),
    "aiwc_job_wait": (_ST, [_VP, ctypes.POINTER(aiwc_metrics)]),
    "aiwc_server_stats": (_ST, [_VP, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "aiwc_server_destroy": (_ST, [_VP]),
}

LIB_PATH = _build.LIB
if not os.path.exists(LIB_PATH):
    raise ImportError(f"libaiwc.so is not built ({LIB_PATH}); run `python -m paper_1805_04207_gb300._build` "
                      "(the AIWC reduction has no CPU fallback)")
lib = ctypes.CDLL(LIB_PATH)
for _name, (_res, _args) in SIGNATURES.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class AiwcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(status: int, handle=None):
    if status != AIWC_OK:
        raise AiwcError(status, (lib.aiwc_last_error(handle) or b"").decode())


# ------------------------------------------------------------------ C names

def aiwc_config_default(**overrides) -> aiwc_config:
    cfg = aiwc_config()
    lib.aiwc_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def aiwc_create(cfg: aiwc_config) -> int:
    h = _VP()
    _check(lib.aiwc_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def aiwc_push_mem(h, ptr: int, n: int, on_device: bool) -> None:
    _check(lib.aiwc_push_mem(h, ptr, n, int(on_device)), h)


def aiwc_push_branch(h, ptr: int, n: int, on_device: bool) -> None:
    _check(lib.aiwc_push_branch(h, ptr, n, int(on_device)), h)


def aiwc_push_instr(h, work_item: int, ptr: int, n: int, on_device: bool) -> None:
    _check(lib.aiwc_push_instr(h, work_item, ptr, n, int(on_device)), h)


def aiwc_push_instr_runs(h, wi_ptr, off_ptr, len_ptr, n_runs, ops_ptr, n_ops, on_device: bool) -> None:
    _check(lib.aiwc_push_instr_runs(h, wi_ptr, off_ptr, len_ptr, n_runs, ops_ptr, n_ops, int(on_device)), h)


def aiwc_push_widths(h, ptr: int, n: int, on_device: bool) -> None:
    _check(lib.aiwc_push_widths(h, ptr, n, int(on_device)), h)


def _from_dict(d: dict) -> aiwc_metrics:
    m = aiwc_metrics()
    for name, _ in METRIC_FIELDS:
        if name == "opcode_hist" or name not in d:
            continue
        if name == "entropy":
            for i, v in enumerate(d[name]):
                m.entropy[i] = v
        else:
            setattr(m, name, d[name])
    return m


def aiwc_aggregate(runs: list, mode: int) -> dict:
    """Sum (AGG_SUM) or median (AGG_MEDIAN) of metric dicts over invocations."""
    arr = (aiwc_metrics * max(1, len(runs)))(*[_from_dict(d) for d in runs])
    out = aiwc_metrics()
    _check(lib.aiwc_aggregate(arr, len(runs), mode, ctypes.byref(out)))
    return _to_dict(out)


def _to_dict(m: aiwc_metrics) -> dict:
    out = {}
    for name, _ in METRIC_FIELDS:
        if name == "opcode_hist":
            continue
        v = getattr(m, name)
        out[name] = list(v) if name == "entropy" else v
    return out


def _hist_ptr(a):
    """The library writes n_opcodes u64 counts through this pointer: only a
    writable, C-contiguous uint64 numpy array (the caller's own) will do."""
    import numpy as np
    if not isinstance(a, np.ndarray) or a.dtype != np.uint64 or not a.flags.c_contiguous or \
            not a.flags.writeable:
        raise ValueError("opcode_hist must be a writable, contiguous uint64 numpy array of n_opcodes")
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def aiwc_compute(h, opcode_hist=None) -> dict:
    """opcode_hist: optional writable uint64 numpy array of n_opcodes."""
    m = aiwc_metrics()
    if opcode_hist is not None:
        m.opcode_hist = _hist_ptr(opcode_hist)
    _check(lib.aiwc_compute(h, ctypes.byref(m)), h)
    return _to_dict(m)


def aiwc_compute_batch(hs, hists=None) -> list[dict]:
    n = len(hs)
    arr = (_VP * n)(*hs)
    outs = (aiwc_metrics * n)()
    if hists is not None:
        for i, hh in enumerate(hists):
            if hh is not None:
                outs[i].opcode_hist = _hist_ptr(hh)
    _check(lib.aiwc_compute_batch(arr, n, outs))
    return [_to_dict(outs[i]) for i in range(n)]


def aiwc_destroy(h) -> None:
    _check(lib.aiwc_destroy(h))


def aiwc_last_error(h=None) -> str:
    return (lib.aiwc_last_error(h) or b"").decode()


def aiwc_device_bytes(h) -> int:
    return int(lib.aiwc_device_bytes(h))


def aiwc_kernel_launches() -> int:
    return int(lib.aiwc_kernel_launches())


def aiwc_set_stage_timing(h, on: bool) -> None:
    _check(lib.aiwc_set_stage_timing(h, int(on)), h)


def aiwc_stage_times(h) -> dict:
    ms = (ctypes.c_double * 32)()
    names = (ctypes.c_char_p * 32)()
    k = lib.aiwc_stage_times(h, ms, names, 32)
    return {names[i].decode(): ms[i] for i in range(k)}


def aiwc_mem_metrics_noalloc(device: int, stream, events_ptr: int, n: int, space_mask: int = 0xF) -> dict:
    """Memory metrics of n device-resident events without any device allocation."""
    m = aiwc_metrics()
    _check(lib.aiwc_mem_metrics_noalloc(device, stream, events_ptr, n, space_mask, ctypes.byref(m)))
    return _to_dict(m)


# ------------------------------------------------------- sharded invocations

def aiwc_shard_route_mem(n_shards: int, events, byte_addresses: int = 0):
    """(routed events, counts per shard) of a host uint8/int64 buffer of 16-byte events (numpy)."""
    import numpy as np
    ev = np.ascontiguousarray(events).view(np.uint8).reshape(-1)
    n = ev.size // 16
    counts = np.zeros(n_shards, dtype=np.uint64)
    n_out = ctypes.c_size_t()
    _check(lib.aiwc_shard_route_mem(n_shards, byte_addresses, ev.ctypes.data, n, None, 0, counts.ctypes.data,
                                    ctypes.byref(n_out)))
    out = np.empty(16 * n_out.value, dtype=np.uint8)
    _check(lib.aiwc_shard_route_mem(n_shards, byte_addresses, ev.ctypes.data, n, out.ctypes.data, n_out.value,
                                    counts.ctypes.data, ctypes.byref(n_out)))
    return out, counts


def aiwc_shard_route_branch(n_shards: int, events):
    """(routed events, counts per shard) of a host buffer of 8-byte branch events (numpy)."""
    import numpy as np
    ev = np.ascontiguousarray(events).view(np.uint8).reshape(-1)
    n = ev.size // 8
    out = np.empty(8 * n, dtype=np.uint8)
    counts = np.zeros(n_shards, dtype=np.uint64)
    _check(lib.aiwc_shard_route_branch(n_shards, ev.ctypes.data, n, out.ctypes.data, counts.ctypes.data))
    return out, counts


def aiwc_shard_route_runs(n_shards: int, run_wi, run_off, run_len, ops):
    """Routed (run_wi u32, run_off u64, run_len u64, ops u16, run_counts, op_counts) of host run tables."""
    import numpy as np
    wi = np.ascontiguousarray(run_wi, dtype=np.uint32)
    off = np.ascontiguousarray(run_off, dtype=np.uint64)
    ln = np.ascontiguousarray(run_len, dtype=np.uint64)
    op = np.ascontiguousarray(ops).view(np.uint16)
    n = wi.size
    o_wi, o_off, o_len = np.empty(n, np.uint32), np.empty(n, np.uint64), np.empty(n, np.uint64)
    total = int(ln.sum()) if n else 0
    o_ops = np.empty(max(total, 1), np.uint16)
    rc, oc = np.zeros(n_shards, np.uint64), np.zeros(n_shards, np.uint64)
    _check(lib.aiwc_shard_route_runs(n_shards, wi.ctypes.data, off.ctypes.data, ln.ctypes.data, n, op.ctypes.data,
                                     op.size, o_wi.ctypes.data, o_off.ctypes.data, o_len.ctypes.data,
                                     o_ops.ctypes.data, rc.ctypes.data, oc.ctypes.data))
    return o_wi, o_off, o_len, o_ops[:total], rc, oc


def aiwc_shard_export(h) -> bytes:
    """This rank's exact distributions as a host blob; the handle is reset."""
    size = ctypes.c_size_t()
    _check(lib.aiwc_shard_export(h, None, 0, ctypes.byref(size)), h)
    buf = ctypes.create_string_buffer(size.value)
    _check(lib.aiwc_shard_export(h, buf, size.value, ctypes.byref(size)), h)
    return buf.raw


def aiwc_shard_merge(h, blobs, opcode_hist=None) -> dict:
    """Metrics of the invocation whose ranks exported `blobs` (bytes each, in rank order)."""
    n = len(blobs)
    keep = [ctypes.create_string_buffer(b, len(b)) for b in blobs]
    ptrs = (_VP * max(n, 1))(*[ctypes.cast(k, _VP) for k in keep])
    sizes = (ctypes.c_size_t * max(n, 1))(*[len(b) for b in blobs])
    m = aiwc_metrics()
    if opcode_hist is not None:
        m.opcode_hist = _hist_ptr(opcode_hist)
    _check(lib.aiwc_shard_merge(h, ptrs, sizes, n, ctypes.byref(m)), h)
    return _to_dict(m)


# ------------------------------------------------------------------ serving

def aiwc_server_config_default(**overrides) -> aiwc_server_config:
    c = aiwc_server_config()
    lib.aiwc_server_config_default(ctypes.byref(c))
    for k, v in overrides.items():
        setattr(c, k, v)
    return c


def aiwc_server_create(cfg: aiwc_server_config) -> int:
    s = _VP()
    _check(lib.aiwc_server_create(ctypes.byref(cfg), ctypes.byref(s)))
    return s.value


def aiwc_job_open(server, cfg: aiwc_config, reserve_bytes: int):
    """A job handle, or None when the server answers AIWC_EAGAIN."""
    j = _VP()
    st = lib.aiwc_job_open(server, ctypes.byref(cfg), reserve_bytes, ctypes.byref(j))
    if st == AIWC_EAGAIN:
        return None
    _check(st)
    return j.value


def aiwc_job_push_mem(j, ptr, n, on_device):
    _check(lib.aiwc_job_push_mem(j, ptr, n, int(on_device)))


def aiwc_job_push_branch(j, ptr, n, on_device):
    _check(lib.aiwc_job_push_branch(j, ptr, n, int(on_device)))


def aiwc_job_push_widths(j, ptr, n, on_device):
    _check(lib.aiwc_job_push_widths(j, ptr, n, int(on_device)))


def aiwc_job_push_instr_runs(j, wi_ptr, off_ptr, len_ptr, n_runs, ops_ptr, n_ops, on_device):
    _check(lib.aiwc_job_push_instr_runs(j, wi_ptr, off_ptr, len_ptr, n_runs, ops_ptr, n_ops, int(on_device)))


def aiwc_job_finish(j):
    _check(lib.aiwc_job_finish(j))


def aiwc_job_poll(j, opcode_hist=None):
    """The metrics dict once the job is done (the job is then released), else None."""
    m = aiwc_metrics()
    if opcode_hist is not None:
        m.opcode_hist = _hist_ptr(opcode_hist)
    st = lib.aiwc_job_poll(j, ctypes.byref(m))
    if st == AIWC_EAGAIN:
        return None
    _check(st)
    return _to_dict(m)


def aiwc_job_wait(j, opcode_hist=None) -> dict:
    m = aiwc_metrics()
    if opcode_hist is not None:
        m.opcode_hist = _hist_ptr(opcode_hist)
    _check(lib.aiwc_job_wait(j, ctypes.byref(m)))
    return _to_dict(m)


def aiwc_server_stats(server) -> dict:
    v = [ctypes.c_uint64() for _ in range(4)]
    _check(lib.aiwc_server_stats(server, *[ctypes.byref(x) for x in v]))
    return dict(zip(("admitted", "rejected", "completed", "device_bytes"), (x.value for x in v)))


def aiwc_server_destroy(server) -> None:
    _check(lib.aiwc_server_destroy(server))


from .api import Characterizer, characterize, compute_batch  # noqa: E402,F401
