"""The C ABI without a GPU: the library loads, exports every function the
header declares, the Python binding's struct layouts match the header, and
argument errors are reported without touching a device."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2511_01235_gb300 import build_ext, native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "maxflow.h")


@pytest.fixture(scope="module")
def lib():
    build_ext.build()
    return native.load()


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(maxflow_[a-z_]+)\s*\(", txt)) - {"maxflow_alloc_fn", "maxflow_free_fn"})


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", build_ext.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (maxflow_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)
    assert sorted(native.EXPORTS) == names


def test_struct_layout_matches_header(tmp_path, lib):
    probe = tmp_path / "probe.c"
    probe.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "maxflow.h"
#define F(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
int main(void) {
  printf("graph %zu\nbatch %zu\nopts %zu\nstats %zu\n", sizeof(maxflow_graph), sizeof(maxflow_batch),
         sizeof(maxflow_opts), sizeof(maxflow_stats_t));
  F(maxflow_opts, max_iters); F(maxflow_opts, time_limit_s); F(maxflow_opts, slack_factor);
  F(maxflow_opts, stream); F(maxflow_opts, alloc); F(maxflow_opts, alloc_user);
  F(maxflow_stats_t, iterations); F(maxflow_stats_t, ms_last); F(maxflow_stats_t, value);
  F(maxflow_batch, on_device);
  return 0;
}
''')
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(probe), "-o", str(exe)])
    got = dict(line.rsplit(" ", 1) for line in subprocess.check_output([str(exe)], text=True).splitlines())
    got = {k: int(v) for k, v in got.items()}
    assert got["graph"] == C.sizeof(native.Graph)
    assert got["batch"] == C.sizeof(native.Batch)
    assert got["opts"] == C.sizeof(native.Opts)
    assert got["stats"] == C.sizeof(native.Stats)
    for k, v in got.items():
        if "." in k:
            T, f = k.split(".")
            cls = {"maxflow_opts": native.Opts, "maxflow_stats_t": native.Stats, "maxflow_batch": native.Batch}[T]
            assert getattr(cls, f).offset == v, k


def test_default_opts_and_strerror(lib):
    o = native.maxflow_default_opts()
    assert (o.data_driven, o.fix_steep, o.kernel_cycles, o.slack_min) == (1, 0, 0, 4)
    assert abs(o.slack_factor - 0.25) < 1e-6
    for code in range(8):
        assert native.strerror(code)
    assert native.strerror(native.ERR_INVALID) == "invalid argument"


def test_init_argument_errors_without_gpu(lib):
    g = native.Graph(3, 1, None, None, None)
    h = C.c_void_p()
    assert lib.maxflow_init(C.byref(h), C.byref(g), 0, 2, None) == native.ERR_INVALID   # NULL arrays
    src = np.array([0], np.int32)
    dst = np.array([1], np.int32)
    cap = np.array([1], np.int32)
    g = native.Graph(3, 1, src.ctypes.data, dst.ctypes.data, cap.ctypes.data)
    assert lib.maxflow_init(C.byref(h), C.byref(g), 1, 1, None) == native.ERR_INVALID   # s == t
    assert lib.maxflow_init(C.byref(h), C.byref(g), 0, 3, None) == native.ERR_INVALID   # t out of range
    assert lib.maxflow_init(None, C.byref(g), 0, 2, None) == native.ERR_INVALID
    assert not h.value


def test_calls_on_null_context(lib):
    v = C.c_int64()
    assert lib.maxflow_query(None, C.byref(v), None, None) == native.ERR_STATE
    assert lib.maxflow_update(None, None) == native.ERR_STATE
    lib.maxflow_destroy(None)


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(native, "_lib", None)
    monkeypatch.setattr(build_ext, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        native.load()


def test_kernel_launch_counter_needs_no_gpu(lib):
    # nothing has been launched in a process without a GPU
    assert lib.maxflow_kernel_launches() == 0
    assert native.kernel_launches() == 0


def test_committed_scheduler_weights_fit_the_action_table(lib):
    # the trained network shipped with the library: 16 features in, one
    # predicted log time per action out, trained for the current action table
    import json
    from oracle import mlp_ref
    from paper_2511_01235_gb300 import scheduler as SCH
    with open(SCH.DEFAULT_WEIGHTS) as f:
        doc = json.load(f)
    acts = native.maxflow_sched_actions()
    assert [tuple(a) for a in doc["actions"]] == [tuple(a) for a in acts]
    n_in, H, n_out = doc["n_in"], doc["n_hidden"], doc["n_out"]
    assert n_in == SCH.N_FEATURES == 16 and n_out == len(acts)
    assert len(doc["params"]) == H * n_in + H + H * H + H + n_out * H + n_out
    assert 0 <= SCH.ACTION_PAPER < n_out and 0 <= SCH.ACTION_DEFAULT < n_out
    y, _ = mlp_ref.forward(np.asarray(doc["params"]), np.full((3, n_in), 0.5), n_in, H, n_out)
    assert np.all(np.isfinite(y))


def test_scheduler_action_table():
    # (mode, rounds, KERNEL_CYCLES, cycle divisor, Alg. 3): mode 0 incremental (Alg. 5),
    # mode 1 static re-solve (Alg. 1); rounds 0 = adaptive, cycles 0 = the average degree.
    # Action 0 is the library default, the paper's fixed schedule is one round with
    # the average degree and Alg. 3 after every discharge.
    from paper_2511_01235_gb300 import scheduler as SCH
    acts = native.maxflow_sched_actions()
    assert acts[SCH.ACTION_DEFAULT] == (0, 0, 0, 0, 0)
    assert acts[SCH.ACTION_PAPER] == (0, 1, 0, 0, 1)
    assert (1, 1, 0, 0, 1) in acts                          # the paper's static solve
    assert len(set(acts)) == len(acts) == 20
    statics = [a for a in acts if a[0] == 1]
    assert len(statics) == 4 and all(a[0] in (0, 1) and a[4] in (0, 1) for a in acts)
    assert all(a[1] in (0, 1, 4, 16, 64) and a[2] in (0, 4, 16, 64) and a[3] in (0, 256) for a in acts)
