"""Eviction, restore and the serving loop on the GPU.

An evicted state restored later continues exactly where it stopped: residual
capacities, heights and excesses are bit-identical, and later updates agree
with the oracle.  In the serving loop, every request's answer is the value the
same sequence of batches gives on that graph alone (exact), with the device
budget forcing evictions and restores, with and without overlap; the final
value of each graph agrees with the oracle's max-flow of its final edge set.
"""
import numpy as np
import pytest

import oracle
from paper_2511_01235_gb300 import native
from paper_2511_01235_gb300 import serving as SV
from paper_2511_01235_gb300 import workloads as W

from helpers import slot_dict

pytestmark = pytest.mark.gpu


def _state(S):
    return slot_dict(*S.residual()), [x.copy() for x in S.vertex_state()]


def test_evict_restore_roundtrip_is_exact():
    g = W.erdos_renyi(3000, 20000, seed=401, cap_hi=100)
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    rng = np.random.default_rng(402)
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    b = W.mixed_batch(es, 2000, rng, ins_cap_hi=100)
    es.apply(b.u, b.v, b.cap)
    S.update(b.u, b.v, b.cap)
    value = S.query()[0]
    before_slots, before_vs = _state(S)
    assert S.device_bytes() > 0
    S.evict()
    assert S.device_bytes() == 0
    assert S.query()[0] == value                     # the value survives eviction
    for call in (lambda: S.update(b.u, b.v, b.cap), lambda: S.residual(), lambda: S.vertex_state(),
                 lambda: S.check(), lambda: S.clone(), lambda: native.maxflow_solve_batched([S], None)):
        with pytest.raises(native.MaxflowError) as ei:
            call()
        assert ei.value.code == native.ERR_STATE
    S.evict()                                        # no-op
    S.restore()
    S.restore()                                      # no-op
    after_slots, after_vs = _state(S)
    assert after_slots == before_slots
    for x, y in zip(before_vs, after_vs):
        np.testing.assert_array_equal(x, y)
    for _ in range(3):                               # continues where it stopped
        b = W.mixed_batch(es, 1500, rng, ins_cap_hi=100)
        es.apply(b.u, b.v, b.cap)
        S.update(b.u, b.v, b.cap)
        u2, v2, c2 = es.coo()
        assert S.query()[0] == oracle.maxflow(g.n, u2, v2, c2, g.s, g.t).value
        S.evict()
        S.restore()
    chk = S.check()
    assert chk["pair_violations"] == 0 and chk["excess_mismatch"] == 0 and chk["active"] == 0
    S.close()


def test_restore_after_slack_overflow_keeps_the_grown_layout():
    # insertions beyond the row slack grow the layout on the device; eviction parks the grown layout
    g = W.erdos_renyi(500, 1500, seed=411, cap_hi=50)
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    rng = np.random.default_rng(412)
    cap0 = S.stats()["slot_capacity"]
    for _ in range(4):
        u = rng.integers(0, 8, size=600).astype(np.int32)          # new edges out of a few rows
        v = rng.integers(0, g.n, size=600).astype(np.int32)
        keep = u != v
        u, v = u[keep], v[keep]
        c = rng.integers(1, 51, size=u.size).astype(np.int32)
        es.apply(u, v, c)
        S.update(u, v, c)
        S.evict()
        S.restore()
        u2, v2, c2 = es.coo()
        assert S.query()[0] == oracle.maxflow(g.n, u2, v2, c2, g.s, g.t).value
    assert S.stats()["slot_capacity"] > cap0
    S.close()


def _mix_graphs():
    gs = [W.rmat(sc, 8, 0.57, 0.19, 0.19, seed=420 + k, cap_hi=1000) for k, sc in enumerate((10, 11, 12, 12, 13))]
    gs.append(W.erdos_renyi(5000, 40000, seed=430, cap_hi=1000))
    return gs


@pytest.mark.parametrize("overlap", [True, False])
def test_serving_answers_equal_alone_under_a_binding_budget(overlap):
    graphs = _mix_graphs()
    reqs = SV.make_requests(graphs, 60, rate_per_s=400.0, seed=440, size_lo=10, size_hi=5000)
    alone, _ = SV.run_alone(graphs, reqs)
    total = 0
    for g in graphs:                                             # the states' footprints
        S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
        total += S.device_bytes()
        S.close()
    budget = int(0.5 * total)
    srv = SV.Server(graphs, budget_bytes=budget, overlap=overlap, group_blocks=4)
    assert srv.resident_bytes() <= budget
    st = srv.run(reqs)
    assert [r.value for r in reqs] == [alone[k] for k in range(len(reqs))]
    assert st.evictions > 0 and st.restores > 0
    assert st.peak_resident_bytes <= budget
    assert srv.arena.stats()["peak_in_use"] <= budget
    # final states agree with the oracle
    sets = [W.EdgeSet(g.n, g.src, g.dst, g.cap) for g in graphs]
    for r in reqs:
        sets[r.graph].apply(r.u, r.v, r.cap)
    for gi, (g, es) in enumerate(zip(graphs, sets)):
        u2, v2, c2 = es.coo()
        assert srv.solvers[gi].query()[0] == oracle.maxflow(g.n, u2, v2, c2, g.s, g.t).value, gi
    s = st.summary()
    assert s["p50_ms"] > 0 and s["p99_ms"] >= s["p50_ms"]
    srv.close()
