"""CPU oracle for dynamic max-flow -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
import this package.  The CUDA library never imports, links or runs it, and
it shares no code with the CUDA path.  This module only marshals arguments
into the plain C implementation in oracle.c (see its header for what each
function follows in the paper and which readings it takes).

Parity pins (tests/test_oracle.py): brute-force min-cut enumeration on tiny
graphs, scipy's independent max-flow, an independent Edmonds-Karp, closed
forms, flow invariants, scipy shortest paths for the heights, hand-derived
fixtures in tests/golden/ for the batch repair and for single steps of
Alg. 2 / Alg. 3 and their pull mirrors, and agreement of the sequential
push-relabel restatement with Dinic on random graphs and batches.
tests/test_oracle_mutations.py plants plausible mistakes in copies of
oracle.c (loaded through MAXFLOW_ORACLE_LIB) and checks that a pin fails.
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


def library_path() -> str:
    """The shared library the wrappers call: liboracle.so built from oracle.c,
    or the prebuilt file named by MAXFLOW_ORACLE_LIB (the mutation tests build
    copies of oracle.c with one planted mistake and point this at them)."""
    return os.environ.get("MAXFLOW_ORACLE_LIB") or _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.environ.get("MAXFLOW_ORACLE_LIB"):
        build()
    L = C.CDLL(library_path())
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
    L.orc_rs_saturate_sink.restype = None
    L.orc_rs_saturate_sink.argtypes = [vp, C.c_int32]
    L.orc_rs_heights_side.restype = None
    L.orc_rs_heights_side.argtypes = [vp, C.c_int32, C.c_int32, vp, C.c_int]
    L.orc_rs_pull_heights.restype = None
    L.orc_rs_pull_heights.argtypes = [vp, C.c_int32, C.c_int32, vp, C.c_int, vp]
    L.orc_rs_pull_value.restype = C.c_int64
    L.orc_rs_pull_value.argtypes = [vp, C.c_int32]
    L.orc_rs_push_side.restype = C.c_int
    L.orc_rs_push_side.argtypes = [vp, C.c_int32, C.c_int32, vp, C.c_int, C.c_int32, C.c_int64]
    L.orc_rs_pull_relabel.restype = C.c_int
    L.orc_rs_pull_relabel.argtypes = [vp, C.c_int32, C.c_int32, vp, C.c_int, C.c_int32, C.c_int64, vp]
    L.orc_rs_cut_side.restype = None
    L.orc_rs_cut_side.argtypes = [vp, vp]
    L.orc_rs_saturate_cut.restype = None
    L.orc_rs_saturate_cut.argtypes = [vp, vp]
    L.orc_rs_set_heights.restype = None
    L.orc_rs_set_heights.argtypes = [vp, i32p]
    L.orc_rs_discharge.restype = C.c_int64
    L.orc_rs_discharge.argtypes = [vp, C.c_int32, C.c_int32, vp]
    L.orc_rs_remove_invalid.restype = None
    L.orc_rs_remove_invalid.argtypes = [vp, C.c_int32, C.c_int32]
    L.orc_rs_pull_discharge.restype = None
    L.orc_rs_pull_discharge.argtypes = [vp, C.c_int32, C.c_int32]
    L.orc_rs_pull_remove_invalid.restype = None
    L.orc_rs_pull_remove_invalid.argtypes = [vp, C.c_int32, C.c_int32]
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

    # ---- single steps from heights the caller sets ----

    def set_heights(self, h):
        h = _a32(h)
        if h.shape != (self.n,) or h.min() < 0 or h.max() > self.n:
            raise ValueError("heights must be n values in [0, n]")
        self._L.orc_rs_set_heights(self._h, h)

    def discharge(self, u, kernel_cycles):
        """Alg. 2 on vertex u for kernel_cycles cycles; returns (pushes, relabels)."""
        rl = np.zeros(1, np.int64)
        pu = self._L.orc_rs_discharge(self._h, int(u), int(kernel_cycles), _ptr(rl))
        return int(pu), int(rl[0])

    def remove_invalid(self, s, t):
        """Alg. 3 on every vertex not in {s, t}."""
        self._L.orc_rs_remove_invalid(self._h, s, t)

    def pull_discharge(self, u, kernel_cycles):
        """The mirror of Alg. 2 for a deficient vertex u (R8)."""
        self._L.orc_rs_pull_discharge(self._h, int(u), int(kernel_cycles))

    def pull_remove_invalid(self, s, t):
        """The mirror of Alg. 3 (R8)."""
        self._L.orc_rs_pull_remove_invalid(self._h, s, t)

    # ---- Sec. 5.2.2 (O2) push and pull (readings R8, R9 in oracle.c) ----

    def saturate_sink(self, t):
        self._L.orc_rs_saturate_sink(self._h, t)

    def pull_heights(self, s, t, side=None, want=0):
        h = np.zeros(self.n, np.int32)
        sd = None if side is None else np.ascontiguousarray(side, dtype=np.uint8)
        self._L.orc_rs_pull_heights(self._h, s, t, _ptr(sd), int(want), _ptr(h))
        return h

    def pull_value(self, t):
        return int(self._L.orc_rs_pull_value(self._h, t))

    def push_side(self, s, t, side, want, kernel_cycles, max_iters=1_000_000):
        sd = None if side is None else np.ascontiguousarray(side, dtype=np.uint8)
        if self._L.orc_rs_push_side(self._h, s, t, _ptr(sd), int(want), kernel_cycles, max_iters) != 0:
            raise RuntimeError("sequential push did not converge")

    def pull_relabel(self, s, t, kernel_cycles, side=None, want=0, max_iters=1_000_000):
        it = np.zeros(1, np.int64)
        sd = None if side is None else np.ascontiguousarray(side, dtype=np.uint8)
        if self._L.orc_rs_pull_relabel(self._h, s, t, _ptr(sd), int(want), kernel_cycles, max_iters, _ptr(it)) != 0:
            raise RuntimeError("sequential pull-relabel did not converge")
        return int(it[0])

    def cut_side(self):
        side = np.zeros(self.n, np.uint8)
        self._L.orc_rs_cut_side(self._h, _ptr(side))
        return side

    def saturate_cut(self, side):
        self._L.orc_rs_saturate_cut(self._h, _ptr(np.ascontiguousarray(side, dtype=np.uint8)))

    def static_pull(self, s, t, kernel_cycles):
        """Max flow by pulling only: saturate the edges into t, then pull-relabel
        with roots s (R8); returns the pull value."""
        self.static_init_empty()
        self.saturate_sink(t)
        self.pull_relabel(s, t, kernel_cycles)
        self.pull_heights(s, t)
        return self.pull_value(t)

    def static_init_empty(self):
        """c_f = c, e = 0, h = 0 (Alg. 1's initialisation without the source step)."""
        self.set_flow(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32))

    def static_push_pull(self, s, t, kernel_cycles):
        """Static push-pull (Sec. 5.2.2): saturate the edges out of s and into t,
        then push with the deficient vertices as sinks; returns the value (R3)."""
        self.static_init(s)
        self.saturate_sink(t)
        v, _, _, _ = self.push_relabel(s, t, kernel_cycles)
        return v

    def push_pull_update(self, s, t, u, v, c, kernel_cycles):
        """The dynamic push-pull of Sec. 5.2.2 on a solved state: the sides of the
        last cut, the batch (Alg. 5), saturation across the cut, push
        on T and pull on S with side-limited roots, then a final push solve (R9)."""
        side = self.cut_side()
        side[s], side[t] = 0, 1
        self.apply(s, u, v, c)
        self.saturate_cut(side)
        self.push_side(s, t, side, 1, kernel_cycles)
        self.pull_relabel(s, t, kernel_cycles, side=side, want=0)
        val, _, _, _ = self.push_relabel(s, t, kernel_cycles)
        return val

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
