"""ctypes binding of the C ABI in include/maxflow.h.

Argument marshalling only: every step of the solver runs in the CUDA library
(paper_2511_01235_gb300/_build/libmaxflow_gb300.so).  If that library is
missing, importing the solver raises at once -- there is no CPU fallback.

The module-level functions carry the C names (maxflow_init, maxflow_update,
maxflow_query, ...); `Solver` is a small object wrapper over them.  Device
memory comes from PyTorch's caching allocator through the allocator
callbacks of maxflow_opts, and work is issued on a torch CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build_ext

OK = 0
ERR_INVALID = 1
ERR_OOM = 2
ERR_CUDA = 3
ERR_NOT_CONVERGED = 4
ERR_STATE = 5
ERR_INTERNAL = 6
ERR_TOO_LARGE = 7


class MaxflowError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (status {code})")


class Graph(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int64), ("src", C.c_void_p), ("dst", C.c_void_p),
                ("cap", C.c_void_p)]


class Batch(C.Structure):
    _fields_ = [("count", C.c_int64), ("u", C.c_void_p), ("v", C.c_void_p), ("new_cap", C.c_void_p),
                ("on_device", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Opts(C.Structure):
    _fields_ = [("kernel_cycles", C.c_int32), ("data_driven", C.c_int32), ("fix_steep", C.c_int32),
                ("grid_blocks", C.c_int32), ("max_iters", C.c_int64), ("time_limit_s", C.c_double),
                ("wait_limit_s", C.c_double), ("slack_factor", C.c_float), ("slack_min", C.c_int32),
                ("device", C.c_int32), ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_user", C.c_void_p)]


class ArenaStats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("capacity", "in_use", "peak_in_use", "free_total", "largest_free",
                                          "free_blocks", "overflow_in_use", "overflow_peak", "fallbacks", "failed")]


class Stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("m_edges", C.c_int64), ("slots", C.c_int64), ("slot_capacity", C.c_int64),
                ("kernel_cycles", C.c_int32), ("grid_blocks", C.c_int32), ("block_threads", C.c_int32),
                ("blocks_per_sm", C.c_int32),
                ("solves", C.c_int64), ("updates", C.c_int64), ("rebuilds", C.c_int64),
                ("iterations", C.c_int64), ("bfs_levels", C.c_int64), ("pushes", C.c_int64),
                ("relabels", C.c_int64), ("steep_fixes", C.c_int64),
                ("active_first", C.c_int64), ("active_total", C.c_int64),
                ("bytes_bfs", C.c_int64), ("bytes_discharge", C.c_int64), ("bytes_fix", C.c_int64),
                ("bytes_worklist", C.c_int64), ("bytes_apply", C.c_int64),
                ("ms_last", C.c_double), ("ms_bfs", C.c_double), ("ms_discharge", C.c_double),
                ("ms_fix", C.c_double), ("ms_worklist", C.c_double), ("ms_apply", C.c_double),
                ("value", C.c_int64), ("ms_kernel", C.c_double), ("barriers", C.c_int64),
                ("discharge_rounds", C.c_int64), ("rounds", C.c_int32), ("reserved0", C.c_int32),
                ("ms_update", C.c_double), ("us_discharge_cta_rows", C.c_double),
                ("us_discharge_warp_rows", C.c_double), ("us_discharge_thread_rows", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ["maxflow_build_layout", "maxflow_kernel_launches", "maxflow_default_opts", "maxflow_init",
           "maxflow_update", "maxflow_query", "maxflow_resolve_static",
           "maxflow_get_flow", "maxflow_stats", "maxflow_destroy", "maxflow_strerror", "maxflow_set_flow",
           "maxflow_apply", "maxflow_global_relabel", "maxflow_resolve", "maxflow_get_residual",
           "maxflow_get_vertex_state", "maxflow_check", "maxflow_global_relabel_noalloc", "maxflow_trace",
           "maxflow_trace_work",
           "maxflow_set_kernel_cycles", "maxflow_clone", "maxflow_set_rounds", "maxflow_sched_actions",
           "maxflow_features", "maxflow_run_action", "maxflow_update_scheduled", "maxflow_mlp_create",
           "maxflow_mlp_destroy", "maxflow_mlp_shape", "maxflow_mlp_get_params", "maxflow_mlp_set_params",
           "maxflow_mlp_forward", "maxflow_mlp_grad", "maxflow_mlp_train", "maxflow_set_tuning",
           "maxflow_solve_batched", "maxflow_device_bytes", "maxflow_evict", "maxflow_restore",
           "maxflow_set_stream", "maxflow_reserve_batch",
           "maxflow_arena_create", "maxflow_arena_destroy", "maxflow_arena_alloc", "maxflow_arena_free",
           "maxflow_arena_stats", "maxflow_arena_fits", "maxflow_evicted_sizes",
           "maxflow_resolve_static_pp", "maxflow_resolve_static_pull", "maxflow_update_pp",
           "maxflow_set_bfs_switch", "maxflow_test_stalled_barrier", "maxflow_set_requeue",
           "maxflow_set_cycle_div", "maxflow_set_fix_steep", "maxflow_set_bfs_tail", "maxflow_checkpoint",
           "maxflow_rollback"]

TRACE_NAMES = ["start", "prologue", "batch_validated", "batch_located", "room_checked", "capacities_changed",
               "iteration_start", "bfs_roots", "bfs_level", "worklist", "discharge", "end", "bfs_bottom_up_first",
               "bfs_cta_join", "bfs_items_split"]

_lib = None


def lib_path() -> str:
    return build_ext.LIB


def load(build_if_missing: bool = False):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = build_ext.LIB
    if not os.path.exists(path):
        if build_if_missing:
            build_ext.build()
        else:
            raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = C.CDLL(path)
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    P = C.POINTER
    L.maxflow_default_opts.argtypes = [P(Opts)]
    L.maxflow_default_opts.restype = None
    L.maxflow_init.argtypes = [P(vp), P(Graph), i32, i32, P(Opts)]
    L.maxflow_update.argtypes = [vp, P(Batch)]
    L.maxflow_apply.argtypes = [vp, P(Batch)]
    L.maxflow_query.argtypes = [vp, P(i64), vp, P(i64)]
    L.maxflow_resolve_static.argtypes = [vp]
    L.maxflow_resolve.argtypes = [vp]
    L.maxflow_global_relabel.argtypes = [vp]
    L.maxflow_get_flow.argtypes = [vp, P(i64), vp, vp, vp, vp]
    L.maxflow_get_residual.argtypes = [vp, P(i64), vp, vp, vp, vp]
    L.maxflow_get_vertex_state.argtypes = [vp, vp, vp]
    L.maxflow_set_flow.argtypes = [vp, i64, vp, vp, vp]
    L.maxflow_stats.argtypes = [vp, P(Stats)]
    L.maxflow_check.argtypes = [vp, vp]
    L.maxflow_trace.argtypes = [vp, vp, vp, i32, P(i32)]
    L.maxflow_trace_work.argtypes = [vp, vp, vp, vp, vp, i32, P(i32)]
    L.maxflow_set_kernel_cycles.argtypes = [vp, i32]
    L.maxflow_set_rounds.argtypes = [vp, i32]
    L.maxflow_set_requeue.argtypes = [vp, i32]
    L.maxflow_set_cycle_div.argtypes = [vp, i32]
    L.maxflow_set_fix_steep.argtypes = [vp, i32]
    L.maxflow_set_bfs_tail.argtypes = [vp, i32]
    L.maxflow_checkpoint.argtypes = [vp]
    L.maxflow_rollback.argtypes = [vp]
    L.maxflow_set_tuning.argtypes = [vp, i32, i32, i32]
    L.maxflow_device_bytes.argtypes = [vp, P(i64)]
    L.maxflow_evict.argtypes = [vp]
    L.maxflow_set_stream.argtypes = [vp, vp]
    L.maxflow_reserve_batch.argtypes = [vp, i64]
    L.maxflow_arena_create.argtypes = [i32, i64, i32, vp, P(vp)]
    L.maxflow_arena_destroy.argtypes = [vp]
    L.maxflow_arena_destroy.restype = None
    L.maxflow_arena_alloc.argtypes = [C.c_size_t, vp, vp]
    L.maxflow_arena_alloc.restype = vp
    L.maxflow_arena_free.argtypes = [vp, C.c_size_t, vp, vp]
    L.maxflow_arena_free.restype = None
    L.maxflow_arena_stats.argtypes = [vp, P(ArenaStats)]
    L.maxflow_arena_fits.argtypes = [vp, vp, i32, P(i32)]
    L.maxflow_evicted_sizes.argtypes = [vp, vp, i32, P(i32)]
    L.maxflow_resolve_static_pp.argtypes = [vp]
    L.maxflow_resolve_static_pull.argtypes = [vp]
    L.maxflow_update_pp.argtypes = [vp, P(Batch), i32]
    L.maxflow_set_bfs_switch.argtypes = [vp, i32, i32]
    L.maxflow_test_stalled_barrier.argtypes = [vp, i32]
    L.maxflow_restore.argtypes = [vp]
    L.maxflow_solve_batched.argtypes = [vp, i32, vp, i32, P(C.c_double)]
    L.maxflow_sched_actions.argtypes = [vp, vp, vp, vp, vp, i32, P(i32)]
    L.maxflow_features.argtypes = [vp, P(Batch), vp]
    L.maxflow_run_action.argtypes = [vp, P(Batch), i32]
    L.maxflow_update_scheduled.argtypes = [vp, P(Batch), vp, P(i32)]
    L.maxflow_mlp_create.argtypes = [P(vp), i32, i32, i32, C.c_uint64, vp]
    L.maxflow_mlp_destroy.argtypes = [vp]
    L.maxflow_mlp_destroy.restype = None
    L.maxflow_mlp_shape.argtypes = [vp, P(i32), P(i32), P(i32), P(i64)]
    L.maxflow_mlp_get_params.argtypes = [vp, vp, i64]
    L.maxflow_mlp_set_params.argtypes = [vp, vp, i64]
    L.maxflow_mlp_forward.argtypes = [vp, vp, i32, vp]
    L.maxflow_mlp_grad.argtypes = [vp, vp, vp, vp, i32, vp, P(C.c_float)]
    L.maxflow_mlp_train.argtypes = [vp, vp, vp, vp, i32, i32, C.c_float, P(C.c_float)]
    L.maxflow_clone.argtypes = [vp, P(vp)]
    L.maxflow_global_relabel_noalloc.argtypes = [i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, i32, vp]
    L.maxflow_destroy.argtypes = [vp]
    L.maxflow_destroy.restype = None
    L.maxflow_strerror.argtypes = [C.c_int]
    L.maxflow_strerror.restype = C.c_char_p
    L.maxflow_kernel_launches.argtypes = []
    L.maxflow_kernel_launches.restype = C.c_int64
    L.maxflow_build_layout.argtypes = [C.c_int32, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_float,
                                       C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p]
    for name in EXPORTS:
        if name not in ("maxflow_kernel_launches", "maxflow_default_opts", "maxflow_destroy", "maxflow_strerror",
                        "maxflow_mlp_destroy", "maxflow_arena_destroy", "maxflow_arena_alloc", "maxflow_arena_free"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def strerror(code: int) -> str:
    try:
        return load().maxflow_strerror(int(code)).decode()
    except ImportError:
        return f"status {code}"


def build_layout(n, src, dst, cap, slack_factor: float = 0.25, slack_min: int = 4) -> dict:
    """The residual Bi-CSR maxflow_init would build (maxflow_build_layout), on the host."""
    L = load()
    src, dst, cap = _i32(src), _i32(dst), _i32(cap)
    S = np.zeros(1, np.int64)
    args = (int(n), int(src.size), _p(src), _p(dst), _p(cap), float(slack_factor), int(slack_min))
    _check(L.maxflow_build_layout(*args, _p(S), None, None, None, None, None, None), "maxflow_build_layout")
    out = {"off": np.zeros(int(n) + 1, np.int32), "deg": np.zeros(int(n), np.int32)}
    for k in ("dst", "cap", "rev", "pcap"):
        out[k] = np.zeros(int(S[0]), np.int32)
    _check(L.maxflow_build_layout(*args, _p(S), _p(out["off"]), _p(out["deg"]), _p(out["dst"]), _p(out["cap"]),
                                  _p(out["rev"]), _p(out["pcap"])), "maxflow_build_layout")
    return out


def kernel_launches() -> int:
    """Kernels the library has launched in this process (maxflow_kernel_launches)."""
    return int(load().maxflow_kernel_launches())


def _check(rc: int, where: str):
    if rc != OK:
        raise MaxflowError(rc, where)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _p(a):
    return C.c_void_p(a.ctypes.data) if a is not None and a.size else None


# ---- torch plumbing -----------------------------------------------------------

class _TorchAllocator:
    """Device memory from torch's caching allocator, handed to the library through callbacks."""

    def __init__(self, device: int):
        import torch
        self.torch = torch
        self.device = device

        def _alloc(nbytes, user, stream):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), device=self.device, stream=int(stream or 0)))
            except Exception:
                return None

        def _free(ptr, nbytes, user, stream):
            try:
                torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:
                pass

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


# ---- the C names ---------------------------------------------------------------

def maxflow_default_opts() -> Opts:
    o = Opts()
    load().maxflow_default_opts(C.byref(o))
    return o


def maxflow_init(n, src, dst, cap, s, t, opts: Opts | None = None):
    src, dst, cap = _i32(src), _i32(dst), _i32(cap)
    g = Graph(int(n), int(src.size), _p(src), _p(dst), _p(cap))
    h = C.c_void_p()
    rc = load().maxflow_init(C.byref(h), C.byref(g), int(s), int(t), C.byref(opts) if opts is not None else None)
    _check(rc, "maxflow_init")
    return h


def _batch(u, v, c):
    """A Batch from numpy (host) or torch CUDA tensors (device); returns (batch, keepalive)."""
    if hasattr(u, "is_cuda") and u.is_cuda:
        import torch
        u = u.to(torch.int32).contiguous()
        v = v.to(torch.int32).contiguous()
        c = c.to(torch.int32).contiguous()
        return Batch(int(u.numel()), u.data_ptr(), v.data_ptr(), c.data_ptr(), 1), (u, v, c)
    if hasattr(u, "numpy"):
        u, v, c = u.numpy(), v.numpy(), c.numpy()
    u, v, c = _i32(u), _i32(v), _i32(c)
    return Batch(int(u.size), _p(u), _p(v), _p(c), 0), (u, v, c)


def maxflow_update(h, u, v, c):
    b, keep = _batch(u, v, c)
    _check(load().maxflow_update(h, C.byref(b)), "maxflow_update")


def maxflow_apply(h, u, v, c):
    b, keep = _batch(u, v, c)
    _check(load().maxflow_apply(h, C.byref(b)), "maxflow_apply")


def maxflow_query(h, n: int, side: bool = False, cut: bool = False):
    val = C.c_int64()
    cc = C.c_int64()
    sd = np.zeros(n, np.uint8) if side else None
    rc = load().maxflow_query(h, C.byref(val), _p(sd) if side else None, C.byref(cc) if cut else None)
    _check(rc, "maxflow_query")
    return int(val.value), (sd.astype(bool) if side else None), (int(cc.value) if cut else None)


def maxflow_resolve_static(h):
    _check(load().maxflow_resolve_static(h), "maxflow_resolve_static")


def maxflow_resolve(h):
    _check(load().maxflow_resolve(h), "maxflow_resolve")


def maxflow_global_relabel(h):
    _check(load().maxflow_global_relabel(h), "maxflow_global_relabel")


def maxflow_get_flow(h):
    L = load()
    cnt = C.c_int64(0)
    _check(L.maxflow_get_flow(h, C.byref(cnt), None, None, None, None), "maxflow_get_flow")
    k = int(cnt.value)
    u, v, cap, f = (np.zeros(max(k, 1), np.int32) for _ in range(4))
    cnt = C.c_int64(k)
    _check(L.maxflow_get_flow(h, C.byref(cnt), _p(u), _p(v), _p(cap), _p(f)), "maxflow_get_flow")
    k = int(cnt.value)
    return u[:k], v[:k], cap[:k], f[:k]


def maxflow_get_residual(h):
    L = load()
    cnt = C.c_int64(0)
    _check(L.maxflow_get_residual(h, C.byref(cnt), None, None, None, None), "maxflow_get_residual")
    k = int(cnt.value)
    u, v, cap, cf = (np.zeros(max(k, 1), np.int32) for _ in range(4))
    cnt = C.c_int64(k)
    _check(L.maxflow_get_residual(h, C.byref(cnt), _p(u), _p(v), _p(cap), _p(cf)), "maxflow_get_residual")
    k = int(cnt.value)
    return u[:k], v[:k], cap[:k], cf[:k]


def maxflow_get_vertex_state(h, n: int):
    hh = np.zeros(n, np.int32)
    e = np.zeros(n, np.int64)
    _check(load().maxflow_get_vertex_state(h, _p(hh), _p(e)), "maxflow_get_vertex_state")
    return hh, e


def maxflow_set_flow(h, u, v, f):
    u, v, f = _i32(u), _i32(v), _i32(f)
    _check(load().maxflow_set_flow(h, int(u.size), _p(u), _p(v), _p(f)), "maxflow_set_flow")


def maxflow_stats(h) -> dict:
    s = Stats()
    _check(load().maxflow_stats(h, C.byref(s)), "maxflow_stats")
    return s.as_dict()


def maxflow_check(h) -> dict:
    out = np.zeros(6, np.int64)
    _check(load().maxflow_check(h, _p(out)), "maxflow_check")
    keys = ["pair_violations", "excess_mismatch", "residual_cross_edges", "active", "cut_cap", "value"]
    return {k: int(x) for k, x in zip(keys, out)}


def maxflow_global_relabel_noalloc(n, s, t, off, deg, dst, cf, pcap, e, h, deficit_roots=True, stream=None):
    """Device pointers (ints) in, heights written to h; allocates nothing on the device."""
    return int(load().maxflow_global_relabel_noalloc(int(n), int(s), int(t), off, deg, dst, cf, pcap, e, h,
                                                      int(bool(deficit_roots)), stream))


def maxflow_trace(h, cap: int = 256):
    """(boundary names, microseconds after kernel entry) of the last solve kernel's grid barriers."""
    b = np.zeros(cap, np.int32)
    t = np.zeros(cap, np.float64)
    k = C.c_int32(0)
    _check(load().maxflow_trace(h, _p(b), _p(t), cap, C.byref(k)), "maxflow_trace")
    k = int(k.value)
    return [TRACE_NAMES[i] if 0 <= i < len(TRACE_NAMES) else str(i) for i in b[:k]], t[:k]


def maxflow_trace_work(h, cap: int = 256):
    """Per entry of maxflow_trace: cumulative slots scanned, packed phase info, and when the
    last and the average CTA finished the phase (microseconds after the previous barrier)."""
    sl = np.zeros(cap, np.int64)
    inf = np.zeros(cap, np.int32)
    last = np.zeros(cap, np.float64)
    mean = np.zeros(cap, np.float64)
    k = C.c_int32(0)
    _check(load().maxflow_trace_work(h, _p(sl), _p(inf), _p(last), _p(mean), cap, C.byref(k)),
           "maxflow_trace_work")
    k = int(k.value)
    return sl[:k], inf[:k], last[:k], mean[:k]


def maxflow_set_kernel_cycles(h, k: int):
    _check(load().maxflow_set_kernel_cycles(h, int(k)), "maxflow_set_kernel_cycles")


def maxflow_set_rounds(h, r: int):
    _check(load().maxflow_set_rounds(h, int(r)), "maxflow_set_rounds")


def maxflow_set_tuning(h, thread_max_slots: int, warp_max_slots: int, bfs_item_min_slots: int):
    _check(load().maxflow_set_tuning(h, int(thread_max_slots), int(warp_max_slots), int(bfs_item_min_slots)),
           "maxflow_set_tuning")


def maxflow_solve_batched(solvers, batches=None, group_blocks=8) -> float:
    """One persistent launch over many instances; returns the launch's device ms."""
    hs = (C.c_void_p * len(solvers))(*[s.h.value for s in solvers])
    keep = []
    bp = None
    if batches is not None:
        arr = (Batch * len(solvers))()
        for i, (u, v, c) in enumerate(batches):
            b, k = _batch(u, v, c)
            arr[i] = b
            keep.append(k)
        bp = C.cast(arr, C.c_void_p)
    ms = C.c_double()
    _check(load().maxflow_solve_batched(C.cast(hs, C.c_void_p), len(solvers), bp, int(group_blocks), C.byref(ms)),
           "maxflow_solve_batched")
    return float(ms.value)


def maxflow_clone(h):
    out = C.c_void_p()
    _check(load().maxflow_clone(h, C.byref(out)), "maxflow_clone")
    return out


def maxflow_sched_actions():
    """The fixed action table: list of (mode, rounds, cycles, cycle_div, fix); mode 0 incremental, 1 static."""
    L = load()
    k = C.c_int32(0)
    _check(L.maxflow_sched_actions(None, None, None, None, None, 0, C.byref(k)), "maxflow_sched_actions")
    n = int(k.value)
    mo, ro, cy, dv, fx = (np.zeros(n, np.int32) for _ in range(5))
    _check(L.maxflow_sched_actions(_p(mo), _p(ro), _p(cy), _p(dv), _p(fx), n, C.byref(k)), "maxflow_sched_actions")
    return list(zip(mo.tolist(), ro.tolist(), cy.tolist(), dv.tolist(), fx.tolist()))


def maxflow_features(h, u, v, c) -> np.ndarray:
    b, keep = _batch(u, v, c)
    out = np.zeros(16, np.float32)
    _check(load().maxflow_features(h, C.byref(b), _p(out)), "maxflow_features")
    return out


def maxflow_run_action(h, u, v, c, action: int):
    b, keep = _batch(u, v, c)
    _check(load().maxflow_run_action(h, C.byref(b), int(action)), "maxflow_run_action")


def maxflow_update_scheduled(h, u, v, c, mlp) -> int:
    b, keep = _batch(u, v, c)
    a = C.c_int32(-1)
    _check(load().maxflow_update_scheduled(h, C.byref(b), mlp.h, C.byref(a)), "maxflow_update_scheduled")
    return int(a.value)


class MLP:
    """The scheduler's network on the device (fp32): n_in -> H -> H -> n_out, ReLU."""

    def __init__(self, n_in=16, n_hidden=64, n_out=None, seed=0, stream=None):
        L = load()
        if n_out is None:
            n_out = len(maxflow_sched_actions())
        h = C.c_void_p()
        st = None if stream is None else int(getattr(stream, "cuda_stream", stream))
        _check(L.maxflow_mlp_create(C.byref(h), int(n_in), int(n_hidden), int(n_out), C.c_uint64(seed), st),
               "maxflow_mlp_create")
        self.h = h
        a, b, c, d = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int64()
        _check(L.maxflow_mlp_shape(h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)), "maxflow_mlp_shape")
        self.n_in, self.n_hidden, self.n_out, self.n_params = a.value, b.value, c.value, d.value

    def close(self):
        if getattr(self, "h", None):
            load().maxflow_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def params(self) -> np.ndarray:
        out = np.zeros(self.n_params, np.float32)
        _check(load().maxflow_mlp_get_params(self.h, _p(out), self.n_params), "maxflow_mlp_get_params")
        return out

    @params.setter
    def params(self, p):
        p = np.ascontiguousarray(np.asarray(p, np.float32))
        _check(load().maxflow_mlp_set_params(self.h, _p(p), int(p.size)), "maxflow_mlp_set_params")

    def forward(self, x) -> np.ndarray:
        x = np.ascontiguousarray(np.asarray(x, np.float32)).reshape(-1, self.n_in)
        y = np.zeros((x.shape[0], self.n_out), np.float32)
        _check(load().maxflow_mlp_forward(self.h, _p(x), x.shape[0], _p(y)), "maxflow_mlp_forward")
        return y

    def grad(self, x, target, mask):
        x = np.ascontiguousarray(np.asarray(x, np.float32)).reshape(-1, self.n_in)
        t = np.ascontiguousarray(np.asarray(target, np.float32)).reshape(-1, self.n_out)
        m = np.ascontiguousarray(np.asarray(mask, np.float32)).reshape(-1, self.n_out)
        g = np.zeros(self.n_params, np.float32)
        loss = C.c_float()
        _check(load().maxflow_mlp_grad(self.h, _p(x), _p(t), _p(m), x.shape[0], _p(g), C.byref(loss)),
               "maxflow_mlp_grad")
        return g, float(loss.value)

    def train(self, x, target, mask, steps=500, lr=3e-3) -> float:
        x = np.ascontiguousarray(np.asarray(x, np.float32)).reshape(-1, self.n_in)
        t = np.ascontiguousarray(np.asarray(target, np.float32)).reshape(-1, self.n_out)
        m = np.ascontiguousarray(np.asarray(mask, np.float32)).reshape(-1, self.n_out)
        loss = C.c_float()
        _check(load().maxflow_mlp_train(self.h, _p(x), _p(t), _p(m), x.shape[0], int(steps), float(lr),
                                        C.byref(loss)), "maxflow_mlp_train")
        return float(loss.value)


def maxflow_destroy(h):
    if h:
        load().maxflow_destroy(h)


# ---- object wrapper --------------------------------------------------------------

class Arena:
    """A device-memory arena (maxflow_arena_*) that Solvers can allocate from.

    nbytes are reserved with one cudaMalloc on `device`, or, with `base` (an
    int address, 256-byte aligned), the caller's region is managed instead.
    """

    def __init__(self, nbytes: int, device: int = 0, allow_overflow: bool = True, base: int | None = None):
        L = load()
        h = C.c_void_p()
        _check(L.maxflow_arena_create(int(device), int(nbytes), int(bool(allow_overflow)), base, C.byref(h)),
               "maxflow_arena_create")
        self.h = h
        self.device = int(device)
        self.alloc_fn = ALLOC_FN(C.cast(L.maxflow_arena_alloc, C.c_void_p).value)
        self.free_fn = FREE_FN(C.cast(L.maxflow_arena_free, C.c_void_p).value)

    def alloc(self, nbytes: int) -> int:
        return load().maxflow_arena_alloc(int(nbytes), self.h, None) or 0

    def free(self, ptr: int):
        load().maxflow_arena_free(ptr, 0, self.h, None)

    def fits(self, sizes) -> bool:
        """Would allocations of these sizes, in this order, all be placed now?"""
        a = np.ascontiguousarray(np.asarray(sizes, dtype=np.int64))
        f = C.c_int32(0)
        _check(load().maxflow_arena_fits(self.h, a.ctypes.data if a.size else None, int(a.size), C.byref(f)),
               "maxflow_arena_fits")
        return bool(f.value)

    def stats(self) -> dict:
        st = ArenaStats()
        _check(load().maxflow_arena_stats(self.h, C.byref(st)), "maxflow_arena_stats")
        return {k: int(getattr(st, k)) for k, _ in ArenaStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            load().maxflow_arena_destroy(self.h)
            self.h = None


class Solver:
    """One dynamic max-flow instance on one GPU (thin wrapper over the C calls)."""

    def __init__(self, n, src, dst, cap, s, t, *, kernel_cycles=0, data_driven=True, fix_steep=False,
                 grid_blocks=0, max_iters=0, time_limit_s=0.0, wait_limit_s=0.0, slack_factor=0.25,
                 slack_min=4, device=None, stream=None, torch_alloc=True, arena=None):
        import torch
        load()
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the solver runs on the GPU only")
        self.n = int(n)
        self.s, self.t = int(s), int(t)
        dev = torch.cuda.current_device() if device is None else int(device)
        self.device = dev
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.evicted = False
        o = maxflow_default_opts()
        o.kernel_cycles = int(kernel_cycles)
        o.data_driven = int(bool(data_driven))
        o.fix_steep = int(bool(fix_steep))
        o.grid_blocks = int(grid_blocks)
        o.max_iters = int(max_iters)
        o.time_limit_s = float(time_limit_s)
        o.wait_limit_s = float(wait_limit_s)
        o.slack_factor = float(slack_factor)
        o.slack_min = int(slack_min)
        o.device = dev
        o.stream = int(self.stream.cuda_stream)
        self._alloc = _TorchAllocator(dev) if torch_alloc and arena is None else None
        if arena is not None:
            self._alloc = arena                  # keeps the arena alive as long as the instance
            o.alloc = arena.alloc_fn
            o.free = arena.free_fn
            o.alloc_user = arena.h.value
        elif self._alloc is not None:
            o.alloc = self._alloc.alloc
            o.free = self._alloc.free
        self._opts = o
        self.h = maxflow_init(n, src, dst, cap, s, t, o)

    def close(self):
        if getattr(self, "h", None):
            maxflow_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, u, v, c):
        maxflow_update(self.h, u, v, c)

    def apply(self, u, v, c):
        maxflow_apply(self.h, u, v, c)

    def query(self, side=False, cut=False):
        return maxflow_query(self.h, self.n, side=side, cut=cut)

    @property
    def value(self) -> int:
        return self.query()[0]

    def resolve_static(self):
        maxflow_resolve_static(self.h)

    def resolve(self):
        maxflow_resolve(self.h)

    def global_relabel(self):
        maxflow_global_relabel(self.h)

    def get_flow(self):
        return maxflow_get_flow(self.h)

    def residual(self):
        return maxflow_get_residual(self.h)

    def vertex_state(self):
        return maxflow_get_vertex_state(self.h, self.n)

    def set_flow(self, u, v, f):
        maxflow_set_flow(self.h, u, v, f)

    def stats(self) -> dict:
        return maxflow_stats(self.h)

    def check(self) -> dict:
        return maxflow_check(self.h)

    def trace(self):
        return maxflow_trace(self.h)

    def trace_work(self):
        return maxflow_trace_work(self.h)

    def set_kernel_cycles(self, k: int):
        maxflow_set_kernel_cycles(self.h, k)

    def set_rounds(self, r: int):
        maxflow_set_rounds(self.h, r)

    def set_requeue(self, on: bool):
        _check(load().maxflow_set_requeue(self.h, int(bool(on))), "maxflow_set_requeue")

    def set_cycle_div(self, div: int):
        _check(load().maxflow_set_cycle_div(self.h, int(div)), "maxflow_set_cycle_div")

    def checkpoint(self):
        """Keep a deep copy of the state (replacing an earlier checkpoint)."""
        _check(load().maxflow_checkpoint(self.h), "maxflow_checkpoint")

    def rollback(self):
        """Return to the last checkpoint's state exactly (after a call that failed)."""
        _check(load().maxflow_rollback(self.h), "maxflow_rollback")

    def set_bfs_tail(self, slots: int):
        _check(load().maxflow_set_bfs_tail(self.h, int(slots)), "maxflow_set_bfs_tail")

    def set_fix_steep(self, on: bool):
        _check(load().maxflow_set_fix_steep(self.h, int(bool(on))), "maxflow_set_fix_steep")

    def device_bytes(self) -> int:
        b = C.c_int64()
        _check(load().maxflow_device_bytes(self.h, C.byref(b)), "maxflow_device_bytes")
        return int(b.value)

    def set_stream(self, stream):
        """Issue this instance's later work on `stream` (a torch.cuda.Stream)."""
        _check(load().maxflow_set_stream(self.h, int(stream.cuda_stream)), "maxflow_set_stream")
        self.stream = stream

    def resolve_static_pp(self):
        """Static push-pull (Sec. 5.2.2): saturate out of s and into t, push with deficits as sinks."""
        _check(load().maxflow_resolve_static_pp(self.h), "maxflow_resolve_static_pp")

    def resolve_static_pull(self):
        """Max flow by pull-relabel alone (Sec. 5.2.2): saturate into t, deficits pull from s."""
        _check(load().maxflow_resolve_static_pull(self.h), "maxflow_resolve_static_pull")

    def update_pp(self, u, v, c, stop_after: int = 0):
        """Dynamic push-pull update (Sec. 5.2.2, dyn-pp-str); stop_after 1 or 2 stops early."""
        b, keep = _batch(u, v, c)
        _check(load().maxflow_update_pp(self.h, C.byref(b), int(stop_after)), "maxflow_update_pp")

    def evicted_sizes(self) -> np.ndarray:
        """Sizes of the device allocations held when evicted (what a restore needs at most)."""
        L = load()
        k = C.c_int32(0)
        _check(L.maxflow_evicted_sizes(self.h, None, 0, C.byref(k)), "maxflow_evicted_sizes")
        out = np.zeros(int(k.value), np.int64)
        _check(L.maxflow_evicted_sizes(self.h, out.ctypes.data, int(out.size), C.byref(k)), "maxflow_evicted_sizes")
        return out

    def reserve_batch(self, count: int):
        """Grow the batch scratch for batches of up to `count` updates now."""
        _check(load().maxflow_reserve_batch(self.h, int(count)), "maxflow_reserve_batch")

    def evict(self):
        """Park the state in pinned host memory and release the device memory."""
        _check(load().maxflow_evict(self.h), "maxflow_evict")
        self.evicted = True

    def restore(self):
        _check(load().maxflow_restore(self.h), "maxflow_restore")
        self.evicted = False

    def set_bfs_switch(self, alpha=14, beta=24):
        """Direction-optimising BFS thresholds (alpha = 0: top-down only)."""
        _check(load().maxflow_set_bfs_switch(self.h, int(alpha), int(beta)), "maxflow_set_bfs_switch")

    def set_tuning(self, thread_max_slots=0, warp_max_slots=0, bfs_item_min_slots=0):
        """Work split thresholds; all 0 (the default) restores the library's defaults."""
        maxflow_set_tuning(self.h, thread_max_slots, warp_max_slots, bfs_item_min_slots)

    def features(self, u, v, c) -> np.ndarray:
        return maxflow_features(self.h, u, v, c)

    def run_action(self, u, v, c, action: int):
        maxflow_run_action(self.h, u, v, c, action)

    def update_scheduled(self, u, v, c, mlp: MLP) -> int:
        return maxflow_update_scheduled(self.h, u, v, c, mlp)

    def clone(self) -> "Solver":
        """A deep copy of this instance's device state (same device, stream and allocator)."""
        other = Solver.__new__(Solver)
        other.n, other.s, other.t = self.n, self.s, self.t
        other.device, other.stream = self.device, self.stream
        other.evicted = False
        other._alloc, other._opts = self._alloc, self._opts
        other.h = maxflow_clone(self.h)
        return other
