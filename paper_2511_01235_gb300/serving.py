"""Serving loop: many max-flow states kept in HBM, update requests batched per tick.

A request is one update batch (Sec. 3: a set of capacity changes) for one of
several graphs; its answer is the new max-flow value.  The server keeps each
graph's residual state (Bi-CSR, preflow, labels) resident in device memory and
repairs it incrementally (Alg. 5), so a request costs a dynamic solve, not a
static one.

Continuous batching: at every tick the server takes the oldest waiting request
of each graph (requests of one graph run in arrival order, so each graph's
state sees exactly the sequence it would see alone) and runs them all in one
persistent launch (maxflow_solve_batched).  Requests that arrive while a launch
runs join the next tick.

Admission by memory: the states do not all fit in the device-memory budget.
The budget is one device arena (maxflow_arena_*): every state allocates from
it, so a restore makes no CUDA allocation call (which would serialise it with
the running launch) and the budget is physical.  A request whose graph is
evicted needs its state restored first; the server evicts the least recently
used graphs that are not in the running launch until the state fits, both in
bytes and as a free block large enough for its largest array.  Evictions and
restores of graphs outside the running launch go on a copy stream from the
host thread while a worker thread waits for the launch on the compute stream,
so state traffic overlaps the solve.
"""
from __future__ import annotations

import math
import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import native
from . import workloads as W


@dataclass
class Request:
    graph: int
    u: np.ndarray
    v: np.ndarray
    cap: np.ndarray
    arrival: float                 # seconds from the start of the run
    start: float = math.nan        # tick that ran it
    done: float = math.nan
    value: int | None = None

    @property
    def size(self) -> int:
        return int(self.u.size)


@dataclass
class ServeStats:
    wall_s: float = 0.0
    device_ms: float = 0.0         # sum of the launches' device time
    ticks: int = 0
    instances: int = 0             # requests run
    updates: int = 0               # edge updates in those requests
    evictions: int = 0
    restores: int = 0
    evict_ms: float = 0.0
    restore_ms: float = 0.0
    peak_resident_bytes: int = 0
    arena_fallbacks: int = 0       # allocations the arena could not place (went to cudaMalloc)
    moves: list = field(default_factory=list)   # (kind, graph, bytes, ms, launch running)
    alg_bytes: float = 0.0         # algorithmic bytes of the launches (the solver's traffic model)
    latencies_ms: list = field(default_factory=list)

    def move_summary(self) -> dict:
        """Evictions and restores: count, GB, ms and GB/s, split by whether a launch was running."""
        out = {}
        for kind in ("evict", "restore"):
            for busy in (False, True):
                mv = [m for m in self.moves if m[0] == kind and m[4] == busy]
                if not mv:
                    continue
                gb = sum(m[2] for m in mv) / 1e9
                ms = sum(m[3] for m in mv)
                out[f"{kind}_{'during_launch' if busy else 'idle'}"] = {
                    "count": len(mv), "gb": gb, "ms": ms, "gbs": gb / (ms / 1e3) if ms > 0 else None,
                    "max_ms": max(m[3] for m in mv)}
        return out

    def summary(self) -> dict:
        lat = np.asarray(self.latencies_ms, np.float64)
        return {"requests": int(self.instances), "updates": int(self.updates), "wall_s": self.wall_s,
                "updates_per_s": self.updates / self.wall_s if self.wall_s > 0 else 0.0,
                "requests_per_s": self.instances / self.wall_s if self.wall_s > 0 else 0.0,
                "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
                "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
                "mean_ms": float(lat.mean()) if lat.size else None,
                "device_busy": self.device_ms / (1e3 * self.wall_s) if self.wall_s > 0 else 0.0,
                "ticks": self.ticks, "mean_batch": self.instances / max(1, self.ticks),
                "evictions": self.evictions, "restores": self.restores,
                "evict_ms": self.evict_ms, "restore_ms": self.restore_ms,
                "peak_resident_gb": self.peak_resident_bytes / 2**30, "arena_fallbacks": self.arena_fallbacks,
                "moves": self.move_summary(),
                "alg_gbs": self.alg_bytes / (self.device_ms * 1e6) if self.device_ms > 0 else 0.0}


class Server:
    """Resident max-flow states under a device-memory budget, served by ticks.

    graphs: list of workloads.Graph; budget_bytes: cap on the sum of the
    resident states' device bytes (maxflow_device_bytes).  Creating the server
    solves every graph once (static solve) and evicts least recently used
    states as the budget requires.
    """

    def __init__(self, graphs, budget_bytes: int, group_blocks: int = 8, overlap: bool = True,
                 max_per_tick: int | None = None, log=None, streams=None, solver_factory=None):
        self.arena = None
        if streams is None:
            import torch
            streams = (torch.cuda.Stream(), torch.cuda.Stream())
        if solver_factory is None:
            import torch
            self.arena = native.Arena(int(budget_bytes), device=torch.cuda.current_device(), allow_overflow=True)
            make = lambda *a, **k: native.Solver(*a, arena=self.arena, **k)
        else:
            make = solver_factory
        self.budget = int(budget_bytes)
        self.group_blocks = int(group_blocks)
        self.overlap = bool(overlap)
        self.max_per_tick = max_per_tick
        self.log = log
        self.compute, self.copy = streams
        self.solvers: list[native.Solver] = []
        self.bytes: list[int] = []
        self.last_use: list[int] = []
        self.clock = 0
        self._busy = False
        self.stats = ServeStats()
        for i, g in enumerate(graphs):
            fb = self._fallbacks()
            S = make(g.n, g.src, g.dst, g.cap, g.s, g.t, stream=self.compute)
            self.solvers.append(S)
            self.bytes.append(S.device_bytes())
            self.last_use.append(self._tick_id())
            self._make_room(0, keep={i}, stream=self.compute)
            if self._fallbacks() > fb:            # created outside the arena: move it in
                S.evict()
                self._make_room(self.bytes[i], keep={i}, stream=self.compute, sizes=S.evicted_sizes())
                S.restore()
            if log:
                log(f"  graph {i}: n={g.n} m={g.src.size} value={S.query()[0]} "
                    f"{self.bytes[i] / 2**20:.0f} MiB, resident {self.resident_bytes() / 2**30:.2f} GiB")
        self.initial_values = [S.query()[0] for S in self.solvers]

    # -- bookkeeping -----------------------------------------------------------

    def _tick_id(self):
        self.clock += 1
        return self.clock

    def _fallbacks(self) -> int:
        return self.arena.stats()["fallbacks"] if self.arena is not None else 0

    def _sizes(self, i):
        S = self.solvers[i]
        return S.evicted_sizes() if self.arena is not None and S.evicted else None

    def _fits(self, need, sizes) -> bool:
        if self.resident_bytes() + need > self.budget:
            return False
        return self.arena is None or sizes is None or self.arena.fits(sizes)

    def resident(self, i) -> bool:
        return not self.solvers[i].evicted

    def resident_bytes(self) -> int:
        return sum(b for i, b in enumerate(self.bytes) if self.resident(i))

    def _evict(self, i, stream):
        S = self.solvers[i]
        t0 = time.perf_counter()
        if stream is not S.stream:
            S.set_stream(stream)
        S.evict()
        ms = (time.perf_counter() - t0) * 1e3
        self.stats.evict_ms += ms
        self.stats.evictions += 1
        self.stats.moves.append(("evict", i, self.bytes[i], ms, self._busy))

    def _restore(self, i, stream):
        S = self.solvers[i]
        t0 = time.perf_counter()
        if stream is not S.stream:
            S.set_stream(stream)
        S.restore()
        if S.stream is not self.compute:
            S.set_stream(self.compute)
        self.bytes[i] = S.device_bytes()
        ms = (time.perf_counter() - t0) * 1e3
        self.stats.restore_ms += ms
        self.stats.restores += 1
        self.stats.moves.append(("restore", i, self.bytes[i], ms, self._busy))

    def _make_room(self, need, keep, stream, sizes=None, spare=()) -> bool:
        """Evict LRU states outside `keep` until `need` more bytes fit the budget
        (and, with the arena, allocations of `sizes` would all be placed).  States
        in `spare` (graphs with waiting requests) go last."""
        while not self._fits(need, sizes):
            victims = [j for j in range(len(self.solvers)) if self.resident(j) and j not in keep]
            if not victims:
                return False
            self._evict(min(victims, key=lambda j: (j in spare, self.last_use[j])), stream)
        return True

    # -- one tick --------------------------------------------------------------

    def _admit(self, heads, busy, waiting=()):
        """Pick this tick's requests: oldest first, restoring evicted graphs as memory allows.

        busy: graphs of the launch still running (never evicted).  Each chosen
        instance's batch scratch is grown before the launch, so the resident
        bytes at launch time (scratch included) stay within the budget.
        """
        chosen = []
        for r in sorted(heads, key=lambda r: r.arrival):
            if self.max_per_tick and len(chosen) >= self.max_per_tick:
                break
            i = r.graph
            keep = set(busy) | {r2.graph for r2 in chosen} | {i}
            if not self.resident(i):
                if not self._make_room(self.bytes[i], keep, self.copy, self._sizes(i), spare=waiting):
                    continue                      # waits for memory; younger resident requests may still go
                self._restore(i, self.copy)
            S = self.solvers[i]
            S.reserve_batch(r.size)
            self.bytes[i] = S.device_bytes()
            if not self._make_room(0, keep, self.copy, spare=waiting):
                self._evict(i, self.copy)         # does not fit beside this tick's others: wait
                continue
            chosen.append(r)
        if not chosen and not busy:
            i = min(heads, key=lambda r: r.arrival).graph
            raise ValueError(f"graph {i} needs {self.bytes[i]} bytes, more than the budget {self.budget}")
        return chosen

    def _launch(self, chosen, out):
        try:
            sol = [self.solvers[r.graph] for r in chosen]
            ms = native.maxflow_solve_batched(sol, [(r.u, r.v, r.cap) for r in chosen],
                                              group_blocks=self.group_blocks)
            out["ms"] = ms
        except BaseException as exc:             # re-raised on the host thread
            out["exc"] = exc

    def run(self, requests: list[Request], log=None) -> ServeStats:
        """Serve `requests` (sorted by arrival, arrival times in seconds from now)."""
        st = self.stats
        queues = [deque() for _ in self.solvers]
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        remaining = len(pending)
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        running = None                            # (thread, out, chosen)
        while remaining:
            t = now()
            while pending and pending[0].arrival <= t:
                r = pending.popleft()
                queues[r.graph].append(r)
            busy = set() if running is None else {r.graph for r in running[2]}
            self._busy = running is not None
            heads = [q[0] for i, q in enumerate(queues) if q and i not in busy]
            nxt = None
            if heads and (running is None or self.overlap):
                # with a launch running, only prepare: restore what the next tick will need
                waiting = {i for i, q in enumerate(queues) if q}
                if running is None:
                    nxt = self._admit(heads, busy, waiting)
                else:
                    # restore, in arrival order, every waiting graph that fits
                    # without evicting another graph with waiting requests
                    for r in sorted(heads, key=lambda r: r.arrival):
                        if self.resident(r.graph):
                            continue
                        if not self._make_room(self.bytes[r.graph], busy | waiting, self.copy,
                                               self._sizes(r.graph)):
                            break
                        self._restore(r.graph, self.copy)
            if running is not None:
                th, out, ch = running
                th.join()
                running = None
                if "exc" in out:
                    raise out["exc"]
                t_done = now()
                st.device_ms += out["ms"]
                st.ticks += 1
                for r in ch:
                    queues[r.graph].popleft()
                    S = self.solvers[r.graph]
                    self.bytes[r.graph] = S.device_bytes()      # batch scratch or a grown layout
                    r.value = S.query()[0]
                    if hasattr(S, "stats"):
                        k = S.stats()
                        st.alg_bytes += (k["bytes_bfs"] + k["bytes_discharge"] + k["bytes_fix"] +
                                         k["bytes_worklist"] + k["bytes_apply"])
                    r.done = t_done
                    st.instances += 1
                    st.updates += r.size
                    st.latencies_ms.append((r.done - r.arrival) * 1e3)
                    self.last_use[r.graph] = self._tick_id()
                    remaining -= 1
                continue
            if not nxt:
                if pending and not any(queues):
                    wait = pending[0].arrival - now()
                    if wait > 2e-3:
                        time.sleep(wait - 1e-3)
                continue
            st.peak_resident_bytes = max(st.peak_resident_bytes, self.resident_bytes())
            for r in nxt:
                r.start = now()
                self.last_use[r.graph] = self._tick_id()
            out = {}
            if self.overlap:
                th = threading.Thread(target=self._launch, args=(nxt, out))
                th.start()
            else:
                th = _Done()
                self._launch(nxt, out)
            running = (th, out, nxt)
        st.wall_s = now()
        st.arena_fallbacks = self._fallbacks()
        for i, S in enumerate(self.solvers):
            if self.resident(i):
                self.bytes[i] = S.device_bytes()
        return st

    def close(self):
        for S in self.solvers:
            S.close()
        self.solvers = []
        if self.arena is not None:
            self.arena.close()
            self.arena = None


class _Done:
    def join(self):
        pass


# ---------------------------------------------------------------------------
# workload: graphs and a Poisson stream of mixed update batches
# ---------------------------------------------------------------------------

SERVING_SCALES = (18, 18, 18, 18, 19, 19, 19, 20, 20, 20, 21, 21, 21, 22, 22, 22)


def serving_graphs(scales=SERVING_SCALES, seed0=10):
    """R-MAT graphs (a, b, c = 0.57, 0.19, 0.19; edge factor 16; caps U[1, 1000]), seeds seed0, seed0+1, ..."""
    return [W.rmat(sc, 16, 0.57, 0.19, 0.19, seed=seed0 + k, cap_hi=1000) for k, sc in enumerate(scales)]


def plan_requests(n_graphs, count, rate_per_s, seed=1, size_lo=10, size_hi=100_000):
    """(graph, batch size, arrival) of `count` requests: Poisson arrivals at
    `rate_per_s` (all at 0 when the rate is 0), graphs uniform at random,
    sizes log-uniform in [size_lo, size_hi]."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=count) if rate_per_s > 0 else np.zeros(count)
    arr = np.cumsum(gaps) - gaps[0]
    gi = rng.integers(0, n_graphs, size=count)
    sizes = np.exp(rng.uniform(math.log(size_lo), math.log(size_hi), size=count)).astype(np.int64)
    return [(int(g), int(b), float(a)) for g, b, a in zip(gi, sizes, arr)]


def graph_batches(graph, sizes, seed):
    """One graph's batches, in order, each drawn against the edge set the earlier
    ones left: mixed batches (increases, decreases, insertions, deletions
    40/40/10/10), sizes capped at a quarter of the edges."""
    rng = np.random.default_rng(seed)
    es = W.EdgeSet(graph.n, graph.src, graph.dst, graph.cap)
    out = []
    for B in sizes:
        b = W.mixed_batch(es, max(1, min(int(B), es.m // 4)), rng, ins_cap_hi=1000)
        es.apply(b.u, b.v, b.cap)
        out.append(b)
    return out


def assemble(plan, batches_per_graph):
    """Requests from a plan and each graph's batch list (consumed in plan order)."""
    nxt = [0] * len(batches_per_graph)
    out = []
    for gi, _, arrival in plan:
        b = batches_per_graph[gi][nxt[gi]]
        nxt[gi] += 1
        out.append(Request(gi, b.u, b.v, b.cap, arrival))
    return out


def make_requests(graphs, count, rate_per_s, seed=1, size_lo=10, size_hi=100_000):
    """`count` requests over `graphs` (plan_requests + graph_batches with seed
    (seed, graph index) for each graph's batches)."""
    plan = plan_requests(len(graphs), count, rate_per_s, seed, size_lo, size_hi)
    per = [graph_batches(g, [b for gi, b, _ in plan if gi == k], (seed, k)) for k, g in enumerate(graphs)]
    return assemble(plan, per)


def retime(requests, rate_per_s, seed=2):
    """Same requests, new Poisson arrival times at `rate_per_s` (order kept)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=len(requests))
    arr = np.cumsum(gaps) - gaps[0]
    for r, a in zip(requests, arr):
        r.arrival = float(a)
        r.start = r.done = math.nan
        r.value = None
    return requests


def run_alone(graphs, requests, stream=None):
    """Each graph's requests applied in order by a fresh instance with nothing else running:
    {request index: value} and the device ms of each request."""
    vals, ms = {}, {}
    for gi, g in enumerate(graphs):
        S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t, stream=stream)
        for k, r in enumerate(requests):
            if r.graph != gi:
                continue
            S.update(r.u, r.v, r.cap)
            vals[k] = S.query()[0]
            ms[k] = S.stats()["ms_last"]
        S.close()
    return vals, ms
