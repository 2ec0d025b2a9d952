"""Host logic of the serving loop, with a fake solver (no GPU).

The fake stands in for the library: its "value" is a hash of the batches it
has seen, in order, so a request answered out of its graph's arrival order,
twice, or from the wrong graph's state changes the answer.  The fake launch
records the resident bytes at launch time and marks its instances busy, and
the fake eviction fails if asked to evict a busy instance.
"""
import hashlib
import threading
import time

import numpy as np
import pytest

from paper_2511_01235_gb300 import serving as SV
from paper_2511_01235_gb300 import workloads as W


class FakeSolver:
    def __init__(self, n, src, dst, cap, s, t, stream=None):
        self.n, self.stream = n, stream
        self.evicted = False
        self.busy = False
        self.scratch = 0
        self.h = hashlib.sha1(f"{n}:{int(np.sum(cap))}".encode()).hexdigest()

    def _feed(self, u, v, c):
        batch = hashlib.sha1(np.concatenate([u, v, c]).tobytes()).hexdigest()
        self.h = hashlib.sha1((self.h + batch).encode()).hexdigest()

    def query(self):
        return (int(self.h[:12], 16), None, None)

    def device_bytes(self):
        return 0 if self.evicted else 1000 * self.n + self.scratch

    def update(self, u, v, c):
        assert not self.evicted
        self._feed(u, v, c)

    def reserve_batch(self, count):               # batch scratch: grows, never shrinks, dropped on eviction
        assert not self.evicted
        self.scratch = max(self.scratch, 500 * int(count))

    def set_stream(self, st):
        self.stream = st

    def evict(self):
        assert not self.busy, "evicted an instance of the running launch"
        self.evicted = True
        self.scratch = 0

    def restore(self):
        self.evicted = False

    def close(self):
        pass


class FakeLaunch:
    def __init__(self, server, delay=0.0):
        self.server, self.delay, self.log = server, delay, []
        self.lock = threading.Lock()

    def __call__(self, solvers, batches, group_blocks=8):
        with self.lock:
            assert all(not s.evicted for s in solvers)
            assert all(s.scratch >= 500 * u.size for s, (u, _, _) in zip(solvers, batches))
            self.log.append((len(solvers), self.server.resident_bytes()))
            for s in solvers:
                s.busy = True
        time.sleep(self.delay)
        for s, (u, v, c) in zip(solvers, batches):
            s._feed(u, v, c)
            s.busy = False
        return 0.1


def _graphs(k, seed=1):
    return [W.erdos_renyi(64 + 16 * i, 256 + 32 * i, seed=seed + i, cap_hi=50) for i in range(k)]


def _alone(graphs, reqs):
    out = {}
    for gi, g in enumerate(graphs):
        S = FakeSolver(g.n, g.src, g.dst, g.cap, g.s, g.t)
        for k, r in enumerate(reqs):
            if r.graph == gi:
                S.update(r.u, r.v, r.cap)
                out[k] = S.query()[0]
    return out


@pytest.mark.parametrize("overlap", [False, True])
@pytest.mark.parametrize("budget_frac", [1.0, 0.45, 0.2])
def test_results_equal_alone_and_budget_respected(monkeypatch, overlap, budget_frac):
    graphs = _graphs(6)
    reqs = SV.make_requests(graphs, 120, rate_per_s=4000.0, seed=3, size_lo=1, size_hi=40)
    alone = _alone(graphs, reqs)
    total = sum(1000 * g.n for g in graphs)
    budget = max(int(budget_frac * total), 1000 * max(g.n for g in graphs) + 500 * 40)
    if budget_frac == 1.0:
        budget = total + 500 * 40 * len(graphs)          # everything fits, scratch included
    srv = SV.Server(graphs, budget, overlap=overlap, streams=("compute", "copy"), solver_factory=FakeSolver)
    fake = FakeLaunch(srv, delay=0.002)
    monkeypatch.setattr(SV.native, "maxflow_solve_batched", fake)
    st = srv.run(reqs)
    assert [r.value for r in reqs] == [alone[k] for k in range(len(reqs))]
    assert st.instances == len(reqs) and len(st.latencies_ms) == len(reqs)
    assert all(r.done >= r.arrival and r.start >= r.arrival for r in reqs)
    for _, resident in fake.log:
        assert resident <= budget
    if budget_frac < 1.0:
        assert st.evictions > 0 and st.restores > 0
    else:
        assert st.evictions == 0
    # requests of one graph complete in arrival order
    for gi in range(len(graphs)):
        done = [r.done for r in reqs if r.graph == gi]
        assert done == sorted(done)
    s = st.summary()
    assert s["p50_ms"] <= s["p99_ms"] and s["requests"] == len(reqs)


def test_a_graph_larger_than_the_budget_is_refused(monkeypatch):
    graphs = _graphs(2)
    reqs = SV.make_requests(graphs, 8, rate_per_s=0, seed=4, size_lo=1, size_hi=8)
    srv = SV.Server(graphs, 1000 * graphs[0].n, streams=("a", "b"), solver_factory=FakeSolver)
    monkeypatch.setattr(SV.native, "maxflow_solve_batched", FakeLaunch(srv))
    if not any(r.graph == 1 for r in reqs):
        pytest.skip("no request for the large graph")
    with pytest.raises(ValueError):
        srv.run(reqs)


def test_lru_eviction_order():
    graphs = _graphs(4)
    srv = SV.Server(graphs, 10**12, streams=("a", "b"), solver_factory=FakeSolver)
    srv.last_use = [5, 2, 9, 7]
    srv.budget = srv.resident_bytes() - 1
    assert srv._make_room(0, keep=set(), stream="b")
    assert [srv.resident(i) for i in range(4)] == [True, False, True, True]
    srv.budget = srv.resident_bytes() + 1000 * graphs[1].n - 1
    assert srv._make_room(1000 * graphs[1].n, keep={0}, stream="b")
    assert [srv.resident(i) for i in range(4)] == [True, False, True, False]


def test_request_stream_is_seeded_and_poisson():
    graphs = _graphs(3)
    a = SV.make_requests(graphs, 2000, rate_per_s=500.0, seed=9, size_lo=1, size_hi=30)
    b = SV.make_requests(graphs, 2000, rate_per_s=500.0, seed=9, size_lo=1, size_hi=30)
    assert [(r.graph, r.arrival, r.size) for r in a] == [(r.graph, r.arrival, r.size) for r in b]
    arr = np.array([r.arrival for r in a])
    gaps = np.diff(arr)
    assert arr[0] == 0 and np.all(gaps >= 0)
    assert abs(gaps.mean() * 500.0 - 1.0) < 0.1                  # exponential gaps, mean 1/rate
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.15           # coefficient of variation 1
    sizes = np.array([r.size for r in a])
    assert sizes.min() >= 1 and sizes.max() <= 30
    # every graph's batches, replayed in order on its edge set, are valid update batches
    for gi, g in enumerate(graphs):
        es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
        for r in a:
            if r.graph == gi:
                assert np.all((r.u >= 0) & (r.u < g.n) & (r.v >= 0) & (r.v < g.n) & (r.u != r.v))
                assert np.all(r.cap >= 0)
                es.apply(r.u, r.v, r.cap)
