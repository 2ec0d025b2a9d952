"""CPU oracle for dynamic max-flow -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
import this package.  The CUDA library never imports, links or runs it, and
it shares no code with the CUDA path.  This module only marshals arguments
into the plain C implementation in oracle.c (see its header for what each
function follows in the paper and which readings it takes).

Parity pins (tests/test_oracle.py): brute-force min-cut enumeration on tiny
graphs, scipy's independent max-flow, an independent Edmonds-Karp, closed
forms, flow invariants, scipy shortest paths for the heights, hand-derived
fixtures in tests/golden/ for the batch repair, and agreement of the
sequential push-relabel restatement with Dinic on random graphs and batches.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library with gcc (plain -O2, no -march)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-Wall", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = C.CDLL(_LIB)
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
    u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
    vp = C.c_void_p
    L.orc_merge.restype = C.c_int64
    L.orc_merge.argtypes = [C.c_int32, C.c_int64, i32p, i32p, i32p, i32p, i32p, i64p]
    L.orc_dinic.restype = C.c_int64
    L.orc_dinic.argtypes = [C.c_int32, C.c_int64, i32p, i32p, i32p, C.c_int32, C.c_int32,
                            vp, vp, vp, vp, vp]
    L.orc_edmonds_karp.restype = C.c_int64
    L.orc_edmonds_karp.argtypes = [C.c_int32, C.c_int64, i32p, i32p, i32p, C.c_int32, C.c_int32]
    L.orc_rs_new.restype = vp
    L.orc_rs_new.argtypes = [C.c_int32, C.c_int64, i32p, i32p, i32p]
    L.orc_rs_free.restype = None
    L.orc_rs_free.argtypes = [vp]
    L.orc_rs_set_flow.restype = C.c_int
    L.orc_rs_set_flow.argtypes = [vp, C.c_int64, i32p, i32p, i32p]
    L.orc_rs_static_init.restype = None
    L.orc_rs_static_init.argtypes = [vp, C.c_int32]
    L.orc_rs_heights.restype = None
    L.orc_rs_heights.argtypes = [vp, C.c_int32, C.c_int32, C.c_int, vp]
    L.orc_rs_apply.restype = C.c_int
    L.orc_rs_apply.argtypes = [C.POINTER(vp), C.c_int32, C.c_int64, i32p, i32p, i32p]
    L.orc_rs_recompute_excess.restype = None
    L.orc_rs_recompute_excess.argtypes = [vp]
    L.orc_rs_value.restype = C.c_int64
    L.orc_rs_value.argtypes = [vp, C.c_int32]
    L.orc_rs_push_relabel.restype = C.c_int64
    L.orc_rs_push_relabel.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int64, vp, vp, vp]
    L.orc_rs_num_slots.restype = C.c_int64
    L.orc_rs_num_slots.argtypes = [vp]
    L.orc_rs_n.restype = C.c_int32
    L.orc_rs_n.argtypes = [vp]
    L.orc_rs_get_slots.restype = None
    L.orc_rs_get_slots.argtypes = [vp, vp, vp, vp, vp]
    L.orc_rs_get_vertex.restype = None
    L.orc_rs_get_vertex.argtypes = [vp, vp, vp]
    L.orc_rs_cut.restype = C.c_int64
    L.orc_rs_cut.argtypes = [vp, vp]
    _lib = L
    return L


def _a32(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.int32))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


@dataclass
class FlowResult:
    value: int
    flow: np.ndarray      # per input edge
    smin: np.ndarray      # bool[n]
    smax: np.ndarray      # bool[n]
    cut_cap: int
    phases: int


def merge(n, src, dst, cap):
    """The current graph: self-loops dropped, parallel edges summed, sorted by (u, v)."""
    L = _load()
    src, dst, cap = _a32(src), _a32(dst), _a32(cap)
    m = src.size
    mu = np.zeros(max(m, 1), np.int32)
    mv = np.zeros(max(m, 1), np.int32)
    mc = np.zeros(max(m, 1), np.int64)
    k = L.orc_merge(n, m, src, dst, cap, mu, mv, mc)
    if k < 0:
        raise ValueError("invalid graph")
    return mu[:k].copy(), mv[:k].copy(), mc[:k].copy()


def maxflow(n, src, dst, cap, s, t) -> FlowResult:
    """Maximum flow by Dinic's algorithm, with S_min, S_max and the cut capacity."""
    L = _load()
    src, dst, cap = _a32(src), _a32(dst), _a32(cap)
    m = src.size
    flow = np.zeros(max(m, 1), np.int32)
    smin = np.zeros(n, np.uint8)
    smax = np.zeros(n, np.uint8)
    cut = np.zeros(1, np.int64)
    ph = np.zeros(1, np.int64)
    v = L.orc_dinic(n, m, src, dst, cap, s, t, _ptr(flow), _ptr(smin), _ptr(smax), _ptr(cut), _ptr(ph))
    if v < 0:
        raise ValueError("invalid graph")
    return FlowResult(int(v), flow[:m], smin.astype(bool), smax.astype(bool), int(cut[0]), int(ph[0]))


def maxflow_ek(n, src, dst, cap, s, t) -> int:
    """Maximum flow by Edmonds-Karp on a dense residual matrix (n <= 4096)."""
    L = _load()
    v = L.orc_edmonds_karp(n, len(src), _a32(src), _a32(dst), _a32(cap), s, t)
    if v < 0:
        raise ValueError("invalid graph")
    return int(v)


class Residual:
    """The paper's residual state: slots (u, v) with c(u, v), c_f(u, v), and e, h per vertex."""

    def __init__(self, n, src, dst, cap):
        self._L = _load()
        self.n = int(n)
        h = self._L.orc_rs_new(n, len(src), _a32(src), _a32(dst), _a32(cap))
        if not h:
            raise ValueError("invalid graph")
        self._h = C.c_void_p(h)

    def __del__(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.orc_rs_free(self._h)
            self._h = None

    def set_flow(self, u, v, f):
        rc = self._L.orc_rs_set_flow(self._h, len(u), _a32(u), _a32(v), _a32(f))
        if rc != 0:
            raise ValueError("invalid flow")

    def static_init(self, s):
        self._L.orc_rs_static_init(self._h, s)

    def recompute_excess(self):
        self._L.orc_rs_recompute_excess(self._h)

    def heights(self, s, t, deficit_roots=True):
        h = np.zeros(self.n, np.int32)
        self._L.orc_rs_heights(self._h, s, t, int(bool(deficit_roots)), _ptr(h))
        return h

    def apply(self, s, u, v, c):
        rc = self._L.orc_rs_apply(C.byref(self._h), s, len(u), _a32(u), _a32(v), _a32(c))
        if rc != 0:
            raise ValueError("invalid batch")

    def value(self, s):
        return int(self._L.orc_rs_value(self._h, s))

    def push_relabel(self, s, t, kernel_cycles, max_iters=1_000_000):
        it = np.zeros(1, np.int64)
        pu = np.zeros(1, np.int64)
        rl = np.zeros(1, np.int64)
        v = self._L.orc_rs_push_relabel(self._h, s, t, kernel_cycles, max_iters, _ptr(it), _ptr(pu), _ptr(rl))
        if v < 0 and v == -1:
            raise RuntimeError("sequential push-relabel did not converge")
        return int(v), int(it[0]), int(pu[0]), int(rl[0])

    def slots(self):
        K = int(self._L.orc_rs_num_slots(self._h))
        u = np.zeros(K, np.int32)
        v = np.zeros(K, np.int32)
        cap = np.zeros(K, np.int64)
        cf = np.zeros(K, np.int64)
        self._L.orc_rs_get_slots(self._h, _ptr(u), _ptr(v), _ptr(cap), _ptr(cf))
        return u, v, cap, cf

    def vertex(self):
        e = np.zeros(self.n, np.int64)
        h = np.zeros(self.n, np.int32)
        self._L.orc_rs_get_vertex(self._h, _ptr(e), _ptr(h))
        return e, h

    def cut(self):
        bad = np.zeros(1, np.int64)
        c = self._L.orc_rs_cut(self._h, _ptr(bad))
        return int(c), int(bad[0])
