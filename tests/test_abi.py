"""The C-ABI library loads, exports every entry point include/*.h declares, and
its structs have the layout the Python binding assumes (no GPU needed)."""
from __future__ import annotations

import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(aiwc_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_builds_and_loads():
    import __graft_entry__
    path = __graft_entry__._builder().build()
    assert os.path.exists(path)
    ctypes.CDLL(path)


def test_every_declared_symbol_is_exported():
    import paper_1805_04207_gb300 as P
    declared = _declared_functions()
    assert {"aiwc_create", "aiwc_push_mem", "aiwc_push_branch", "aiwc_push_instr", "aiwc_compute"} <= declared
    for name in declared:
        assert hasattr(P.lib, name), name
    # the binding wraps every declared entry point with the same name
    assert declared <= set(P.SIGNATURES), declared - set(P.SIGNATURES)
    out = subprocess.run(["nm", "-D", "--defined-only", P.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (aiwc_\w+)", out))
    assert declared <= exported, declared - exported


def test_struct_layout_matches_header(tmp_path):
    import paper_1805_04207_gb300 as P
    src = tmp_path / "layout.c"
    fields_m = [n for n, _ in P.METRIC_FIELDS]
    fields_c = [n for n, _ in P.aiwc_config._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "aiwc.h"', "int main(void){",
             'printf("%zu %zu\\n", sizeof(aiwc_metrics), sizeof(aiwc_config));']
    lines += [f'printf("%zu\\n", offsetof(aiwc_metrics, {f}));' for f in fields_m]
    lines += [f'printf("%zu\\n", offsetof(aiwc_config, {f}));' for f in fields_c]
    lines += ['printf("%zu %zu\\n", sizeof(aiwc_mem_event), sizeof(aiwc_branch_event));', "return 0;}"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    vals = [int(v) for v in vals]
    assert vals[0] == ctypes.sizeof(P.aiwc_metrics) and vals[1] == ctypes.sizeof(P.aiwc_config)
    k = 2
    for f in fields_m:
        assert vals[k] == getattr(P.aiwc_metrics, f).offset, f
        k += 1
    for f in fields_c:
        assert vals[k] == getattr(P.aiwc_config, f).offset, f
        k += 1
    assert vals[k:] == [16, 8]


def test_config_defaults_are_the_papers():
    import paper_1805_04207_gb300 as P
    c = P.aiwc_config_default()
    assert (c.history_len, c.cover_num, c.cover_den, c.space_mask, c.n_opcodes) == (16, 9, 10, 0xF, 65535)


def test_invalid_config_rejected_without_touching_a_device():
    import paper_1805_04207_gb300 as P
    for bad in (dict(history_len=0), dict(history_len=32), dict(cover_num=11), dict(cover_den=0),
                dict(n_opcodes=0), dict(precision=2), dict(max_work_items=(1 << 32) + 1)):
        with pytest.raises(P.AiwcError) as e:
            P.aiwc_create(P.aiwc_config_default(**bad))
        assert e.value.status == P.AIWC_EINVAL


def test_null_arguments_are_errors_not_crashes():
    import paper_1805_04207_gb300 as P
    assert P.lib.aiwc_create(None, None) == P.AIWC_EINVAL
    assert P.lib.aiwc_push_mem(None, None, 0, 0) == P.AIWC_EINVAL
    assert P.lib.aiwc_compute(None, None) == P.AIWC_EINVAL
    assert P.lib.aiwc_destroy(None) == P.AIWC_OK


def test_product_package_does_not_reach_the_oracle():
    pkg = os.path.join(ROOT, "paper_1805_04207_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if os.path.isfile(path) and path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            text = open(path).read()
            assert "import oracle" not in text and "from oracle" not in text, path
            assert "aiwc_oracle" not in text and "liboracle" not in text, path


def test_import_fails_loudly_without_the_library(tmp_path):
    """A copy of the package whose library was never built refuses to import:
    there is no CPU fallback to land on."""
    import shutil
    import subprocess
    import sys
    dst = tmp_path / "paper_1805_04207_gb300"
    shutil.copytree(os.path.join(ROOT, "paper_1805_04207_gb300"), dst,
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    r = subprocess.run([sys.executable, "-c", "import paper_1805_04207_gb300"], cwd=tmp_path,
                       capture_output=True, text=True, env={**os.environ, "PYTHONPATH": str(tmp_path)})
    assert r.returncode != 0
    assert "libaiwc.so is not built" in r.stderr


def test_binding_passes_only_the_callers_own_buffers():
    """The binding hands the library the caller's buffer itself, never a
    temporary copy that would be freed before the library reads it."""
    import numpy as np
    import torch

    from paper_1805_04207_gb300.api import _ptr
    a = np.arange(8, dtype=np.int64)
    assert _ptr(a) == (a.ctypes.data, False)
    t = torch.arange(8, dtype=torch.int64)
    assert _ptr(t) == (t.data_ptr(), False)
    for bad in ([1, 2, 3], a[::2], t[::2]):
        with pytest.raises(ValueError):
            _ptr(bad)


def test_histogram_buffer_is_checked_before_the_library_writes_it():
    import numpy as np

    import paper_1805_04207_gb300 as P
    assert P._hist_ptr(np.zeros(4, dtype=np.uint64))
    for bad in (np.zeros(4, dtype=np.int32), np.zeros(8, dtype=np.uint64)[::2], [0, 0, 0]):
        with pytest.raises(ValueError):
            P._hist_ptr(bad)
    ro = np.zeros(4, dtype=np.uint64)
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        P._hist_ptr(ro)


def test_binding_counts_records_by_bytes_and_checks_table_widths():
    import numpy as np
    import torch

    from paper_1805_04207_gb300.api import _elements, _records
    assert _records(torch.zeros((5, 2), dtype=torch.int64), 16, "m") == 5
    assert _records(torch.zeros(80, dtype=torch.uint8), 16, "m") == 5
    assert _records(np.zeros(3, dtype=np.int64), 8, "b") == 3
    with pytest.raises(ValueError):
        _records(torch.zeros(3, dtype=torch.int64), 16, "m")  # 24 bytes: not whole 16-byte events
    assert _elements(torch.zeros(7, dtype=torch.int32), 4, "run_wi") == 7
    with pytest.raises(ValueError):
        _elements(torch.zeros(7, dtype=torch.int64), 4, "run_wi")  # a 64-bit run table would be misread
    with pytest.raises(ValueError):
        _elements(np.zeros(7, dtype=np.int32), 2, "opcodes")


def test_push_wrappers_pass_record_counts(monkeypatch):
    """With the C calls replaced by recorders (no device needed), pushing a
    synthetic invocation hands the library each stream's record count and
    the tensors' own addresses."""
    import torch

    import synth
    from paper_1805_04207_gb300 import api
    calls = []
    for name in ("aiwc_push_mem", "aiwc_push_branch", "aiwc_push_widths"):
        monkeypatch.setattr(api, name, lambda h, p, n, dev, _n=name: calls.append((_n, p, n, dev)))
    monkeypatch.setattr(api, "aiwc_push_instr_runs",
                        lambda h, pw, po, pl, nr, pp, no, dev: calls.append(("runs", pw, po, pl, nr, pp, no, dev)))
    c = object.__new__(api.Characterizer)
    c.h, c._keep = None, []
    tr = synth.tiny()
    api.push_trace(c, tr)
    got = {k[0]: k for k in calls}
    assert got["aiwc_push_mem"][1:] == (tr.mem.data_ptr(), tr.mem.shape[0], False)
    assert got["aiwc_push_branch"][1:] == (tr.br.data_ptr(), tr.br.shape[0], False)
    assert got["aiwc_push_widths"][1:] == (tr.widths.data_ptr(), tr.widths.shape[0], False)
    r = got["runs"]
    assert r[2:5] == (tr.run_off.data_ptr(), tr.run_len.data_ptr(), tr.run_wi.shape[0])
    assert r[5:] == (tr.ops.data_ptr(), tr.ops.shape[0], False)
    with pytest.raises(ValueError):
        c.push_instr_runs(tr.run_wi, tr.run_off, tr.run_len, tr.ops)  # 64-bit work-item table
    with pytest.raises(ValueError):
        c.push_instr_runs(tr.run_wi.to(torch.int32), tr.run_off[:-1], tr.run_len, tr.ops)


def test_plain_c_client_links_and_runs(tmp_path):
    """The boundary is a C ABI: a C program built against include/aiwc.h and
    linked to libaiwc.so runs the calls that need no device."""
    import paper_1805_04207_gb300 as P
    libdir = os.path.dirname(P.LIB_PATH)
    exe = tmp_path / "c_client"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_client.c"), "-L", libdir, "-laiwc", f"-Wl,-rpath,{libdir}",
                    "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "c client ok"
