"""CPU oracle for the AIWC metrics -- TEST INFRASTRUCTURE ONLY.

Builds ``aiwc_oracle.cpp`` with the host compiler and calls it through
ctypes. Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline leg may import this package; the product path never does.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aiwc_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

METRIC_FIELDS = [
    ("total_instructions", ctypes.c_uint64), ("unique_opcodes", ctypes.c_uint64),
    ("opcode_cover", ctypes.c_uint64), ("work_items", ctypes.c_uint64), ("barriers", ctypes.c_uint64),
    ("itb_count", ctypes.c_uint64), ("itb_min", ctypes.c_uint64), ("itb_max", ctypes.c_uint64),
    ("itb_median_lo", ctypes.c_uint64), ("itb_median_hi", ctypes.c_uint64), ("itb_median", ctypes.c_double),
    ("ipt_count", ctypes.c_uint64), ("ipt_min", ctypes.c_uint64), ("ipt_max", ctypes.c_uint64),
    ("ipt_median_lo", ctypes.c_uint64), ("ipt_median_hi", ctypes.c_uint64), ("ipt_median", ctypes.c_double),
    ("total_reads", ctypes.c_uint64), ("total_writes", ctypes.c_uint64), ("footprint", ctypes.c_uint64),
    ("footprint_cover", ctypes.c_uint64), ("unique_reads", ctypes.c_uint64), ("unique_writes", ctypes.c_uint64),
    ("entropy", ctypes.c_double * 11),
    ("branch_events", ctypes.c_uint64), ("branch_sites", ctypes.c_uint64), ("branch_cover", ctypes.c_uint64),
    ("branch_patterns", ctypes.c_uint64), ("branch_minsum", ctypes.c_uint64), ("albe", ctypes.c_double),
    ("yokota", ctypes.c_double),
    ("unique_rw_ratio", ctypes.c_double), ("reread_ratio", ctypes.c_double), ("rewrite_ratio", ctypes.c_double),
]


class _Metrics(ctypes.Structure):
    _fields_ = METRIC_FIELDS


class _Config(ctypes.Structure):
    _fields_ = [("history_len", ctypes.c_uint32), ("cover_num", ctypes.c_uint32),
                ("cover_den", ctypes.c_uint32), ("n_opcodes", ctypes.c_uint32),
                ("space_mask", ctypes.c_uint32), ("byte_addresses", ctypes.c_uint32),
                ("history_scope", ctypes.c_uint32)]


class OracleInvalidInput(ValueError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (plain g++ -O2)."""
    import fcntl
    os.makedirs(_OUT_DIR, exist_ok=True)
    with _lock, open(os.path.join(_OUT_DIR, ".lock"), "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _bind(lib):
    lib.aiwc_oracle_compute.restype = ctypes.c_int
    lib.aiwc_oracle_compute.argtypes = [
        ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64,
        ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
        ctypes.c_uint64, ctypes.POINTER(_Config), ctypes.POINTER(_Metrics), ctypes.c_void_p]
    lib.aiwc_oracle_simd.restype = None
    lib.aiwc_oracle_simd.argtypes = [ctypes.c_void_p, ctypes.c_uint64] + [ctypes.POINTER(ctypes.c_uint64)] * 4
    lib.aiwc_oracle_count_of_counts.restype = ctypes.c_int64
    lib.aiwc_oracle_count_of_counts.argtypes = [
        ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def build_variant(source: str, out_dir: str, name: str) -> str:
    """Compile an edited copy of the oracle source (used to plant mistakes in tests)."""
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(out_dir, name + ".cpp")
    with open(src, "w") as f:
        f.write(source)
    lib = os.path.join(out_dir, name + ".so")
    subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-o", lib, src], check=True)
    return lib


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _np(t, dtype):
    if t is None:
        return np.zeros(0, dtype=dtype)
    if hasattr(t, "detach"):
        t = t.detach().cpu().contiguous().numpy()
    return np.ascontiguousarray(t).view(dtype) if np.asarray(t).dtype.itemsize == np.dtype(dtype).itemsize \
        else np.ascontiguousarray(t).astype(dtype)


def _mem_bytes(mem):
    if mem is None:
        return np.zeros(0, dtype=np.uint8), 0
    a = mem.detach().cpu().contiguous().numpy() if hasattr(mem, "detach") else np.ascontiguousarray(mem)
    b = np.ascontiguousarray(a).view(np.uint8).reshape(-1)
    assert b.size % 16 == 0
    return b, b.size // 16


def compute(trace, history_len: int = 16, cover_num: int = 9, cover_den: int = 10,
            n_opcodes: int | None = None, space_mask: int = 0xF, want_hist: bool = True,
            lib_path: str | None = None, byte_addresses: int = 0, history_scope: int = 0) -> dict:
    """Metrics of one invocation (a synth.Trace or anything with the same fields).

    byte_addresses=1 counts every byte an access touches as an access of its
    own; history_scope=1 keeps one branch history per (site, work-item).
    """
    lib = _load() if lib_path is None else _bind(ctypes.CDLL(lib_path))
    mem, n_mem = _mem_bytes(trace.mem)
    br = _np(trace.br, np.uint64)
    ops = _np(trace.ops, np.uint16)
    run_wi = _np(trace.run_wi, np.int64).astype(np.uint32)
    run_off = _np(trace.run_off, np.uint64)
    run_len = _np(trace.run_len, np.uint64)
    nop = trace.n_opcodes if n_opcodes is None else n_opcodes
    cfg = _Config(history_len, cover_num, cover_den, nop, space_mask, byte_addresses, history_scope)
    out = _Metrics()
    hist = np.zeros(max(1, nop), dtype=np.uint64)
    rc = lib.aiwc_oracle_compute(mem.ctypes.data, n_mem, br.ctypes.data, br.size, ops.ctypes.data, ops.size,
                                 run_wi.ctypes.data, run_off.ctypes.data, run_len.ctypes.data, run_wi.size,
                                 ctypes.byref(cfg), ctypes.byref(out), hist.ctypes.data if want_hist else None)
    if rc != 0:
        raise OracleInvalidInput("oracle rejected the input")
    res = {}
    for name, _ in METRIC_FIELDS:
        v = getattr(out, name)
        res[name] = list(v) if name == "entropy" else v
    if want_hist:
        res["opcode_hist"] = hist[:nop].copy()
    res.update(simd(getattr(trace, "widths", None), lib))
    res.update(derived(res))
    return res


def simd(widths, lib=None) -> dict:
    """Table I SIMD rows from the per-instruction result widths (Sec. V)."""
    lib = _load() if lib is None else lib
    w = _np(widths, np.uint16)
    c, m, s, q = (ctypes.c_uint64() for _ in range(4))
    lib.aiwc_oracle_simd(w.ctypes.data, w.size, ctypes.byref(c), ctypes.byref(m), ctypes.byref(s), ctypes.byref(q))
    c, m, s, q = c.value, m.value, s.value, q.value
    # population variance (count * sumsq - sum^2) / count^2, numerator in exact integers
    mean = s / c if c else 0.0
    sd = math.sqrt((c * q - s * s) / (c * c)) if c else 0.0
    return {"simd_count": c, "simd_max": m, "simd_sum": s, "simd_sumsq": q, "simd_mean": mean, "simd_sd": sd}


def _div(a, b) -> float:
    # IEEE division as the metric structure defines it: x/0 is inf, 0/0 is NaN
    a, b = float(a), float(b)
    if b == 0.0:
        return math.nan if a == 0.0 else math.copysign(math.inf, a)
    return a / b


def derived(m: dict) -> dict:
    """The derived parallelism quantities of the Kiviat diagrams (Sec. VI)."""
    return {
        "granularity": _div(1, m["work_items"]),
        # 1 / mean ITB, mean ITB = sum of ITB (= total instructions) / number of ITB values
        "barriers_per_instruction": _div(m["itb_count"], m["total_instructions"]),
        "instructions_per_operand": _div(1, m["simd_sum"]),
        "load_imbalance": float(m["ipt_max"] - m["ipt_min"]),
    }


def aggregate(runs: list, mode: str) -> dict:
    """Whole-application view over invocations (Sec. VI): "sum" adds every
    numeric metric; "median" takes each metric's median across the runs (mean
    of the two middle values for real-valued metrics, the lower middle value
    for counts)."""
    out = {}
    for k in runs[0]:
        if k == "opcode_hist":
            continue
        vals = [r[k] for r in runs]
        if k == "entropy":
            cols = list(zip(*vals))
            out[k] = [_agg_real(list(c), mode) for c in cols]
        elif isinstance(vals[0], float):
            out[k] = _agg_real(vals, mode)
        else:
            out[k] = sum(vals) if mode == "sum" else sorted(vals)[(len(vals) - 1) // 2]
    return out


def _agg_real(vals, mode):
    if mode == "sum":
        t = 0.0
        for v in vals:  # in run order
            t += v
        return t
    v = sorted(vals)
    return 0.5 * (v[(len(v) - 1) // 2] + v[len(v) // 2])


def count_of_counts(mem, n: int, space_mask: int = 0xF, lib_path: str | None = None) -> dict:
    """{c: m_c} of the memory accesses grouped by key >> n."""
    lib = _load() if lib_path is None else _bind(ctypes.CDLL(lib_path))
    b, n_mem = _mem_bytes(mem)
    cap = 1 << 16
    while True:
        c = np.zeros(cap, dtype=np.uint64)
        m = np.zeros(cap, dtype=np.uint64)
        w = lib.aiwc_oracle_count_of_counts(b.ctypes.data, n_mem, space_mask, n, c.ctypes.data,
                                            m.ctypes.data, cap)
        if w < 0:
            raise OracleInvalidInput("oracle rejected the input")
        if w <= cap:
            return {int(c[i]): int(m[i]) for i in range(w)}
        cap = int(w)
