"""Many instances in one persistent launch (maxflow_solve_batched), and the
work-split thresholds (maxflow_set_tuning): the values stay those of the
oracle whatever the grouping or the thresholds."""
import numpy as np
import pytest

import oracle
from paper_2511_01235_gb300 import native
from paper_2511_01235_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _instances(count, seed, lo=200, hi=6000):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        kind = i % 3
        if kind == 0:
            g = W.erdos_renyi(n, 8 * n, seed=seed * 100 + i, cap_hi=500)
        elif kind == 1:
            g = W.layered_dag(max(n, 40), seed=seed * 100 + i, cap_hi=500)
        else:
            g = W.geometric(n, seed=seed * 100 + i, cap_hi=500)
        out.append(g)
    return out


@pytest.mark.parametrize("group", [1, 4, 16])
def test_batched_static_matches_oracle(group):
    gs = _instances(12, 5)
    S = [native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t) for g in gs]
    ms = native.maxflow_solve_batched(S, None, group_blocks=group)
    assert ms > 0
    for g, s in zip(gs, S):
        assert s.query()[0] == oracle.maxflow(g.n, g.src, g.dst, g.cap, g.s, g.t).value
        chk = s.check()
        assert chk["active"] == 0 and chk["residual_cross_edges"] == 0 and chk["cut_cap"] == chk["value"]
        s.close()


def test_batched_updates_match_oracle():
    gs = _instances(10, 6)
    S = [native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t) for g in gs]
    rng = np.random.default_rng(7)
    for rep in range(2):
        batches, sets = [], []
        for g in gs:
            es = getattr(g, "_es", None) or W.EdgeSet(g.n, g.src, g.dst, g.cap)
            g._es = es
            b = W.mixed_batch(es, max(1, es.m // 100), rng, ins_cap_hi=500)
            es.apply(b.u, b.v, b.cap)
            batches.append((b.u, b.v, b.cap))
        native.maxflow_solve_batched(S, batches, group_blocks=4)
        for g, s in zip(gs, S):
            u2, v2, c2 = g._es.coo()
            assert s.query()[0] == oracle.maxflow(g.n, u2, v2, c2, g.s, g.t).value
    for s in S:
        s.close()


@pytest.mark.parametrize("tun", [(1, 1, 1), (32, 64, 64), (64, 100000, 100000)])
def test_tuning_thresholds_do_not_change_the_value(tun):
    g = W.rmat(14, 16, 0.57, 0.19, 0.19, seed=41, cap_hi=1000)
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    S.set_tuning(*tun)
    S.resolve_static()
    assert S.query()[0] == oracle.maxflow(g.n, g.src, g.dst, g.cap, g.s, g.t).value
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    b = W.mixed_batch(es, 2000, np.random.default_rng(42), ins_cap_hi=1000)
    es.apply(b.u, b.v, b.cap)
    S.update(b.u, b.v, b.cap)
    u2, v2, c2 = es.coo()
    assert S.query()[0] == oracle.maxflow(g.n, u2, v2, c2, g.s, g.t).value
    S.close()
