"""Pins of the oracle's push and pull (Sec. 5.2.2, O2; readings R8, R9 in oracle.c).

The values are pinned to Dinic (an independent algorithm) on varied graphs;
the steps are pinned by properties the section states: after saturating the
edges across the old cut no residual edge leads from S to T, the push part
touches only T and the pull part only S, and a finished pull leaves no
deficient vertex reachable from s.
"""
import numpy as np
import pytest

import oracle
from paper_2511_01235_gb300 import workloads as W


def _graphs():
    out = []
    for seed in range(12):
        out.append(W.erdos_renyi(80, 400, seed=100 + seed, cap_hi=30))
    out.append(W.rmat(9, 8, 0.57, 0.19, 0.19, seed=7, cap_hi=50))
    out.append(W.layered_dag(200, seed=8, layers=6, fanout=4, cap_hi=40))
    G = W.GridSegmentation(side=16, seed=3, window=4, origin=(4, 4), step=1)
    out.append(G.graph())
    return out


GRAPHS = _graphs()


def _residual_reach(n, u, v, cf, roots):
    """Vertices reachable from roots over slots (u, v) with cf > 0."""
    adj = [[] for _ in range(n)]
    for a, b, c in zip(u, v, cf):
        if c > 0:
            adj[a].append(b)
    seen = np.zeros(n, bool)
    stack = list(roots)
    for r in roots:
        seen[r] = True
    while stack:
        x = stack.pop()
        for y in adj[x]:
            if not seen[y]:
                seen[y] = True
                stack.append(y)
    return seen


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_static_pull_and_static_push_pull_equal_dinic(gi):
    g = GRAPHS[gi]
    want = oracle.maxflow(g.n, g.src, g.dst, g.cap, g.s, g.t).value
    for kc in (1, 3, 16):
        R = oracle.Residual(g.n, g.src, g.dst, g.cap)
        assert R.static_pull(g.s, g.t, kc) == want
        e, _ = R.vertex()
        assert -e[g.s] == want                       # all the flow leaves s
        assert np.all(np.delete(e, [g.s, g.t]) <= 0)  # pulling creates no excess
        R2 = oracle.Residual(g.n, g.src, g.dst, g.cap)
        assert R2.static_push_pull(g.s, g.t, kc) == want


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_finished_pull_leaves_no_reachable_deficit(gi):
    g = GRAPHS[gi]
    R = oracle.Residual(g.n, g.src, g.dst, g.cap)
    R.static_init_empty()
    R.saturate_sink(g.t)
    e0, _ = R.vertex()
    assert np.all(np.delete(e0, [g.t]) <= 0) and e0[g.t] >= 0
    R.pull_relabel(g.s, g.t, 4)
    u, v, cap, cf = R.slots()
    e, _ = R.vertex()
    reach = _residual_reach(g.n, u, v, cf, [g.s])
    deficit = (e < 0) & (np.arange(g.n) != g.s) & (np.arange(g.n) != g.t)
    assert not np.any(reach & deficit)
    assert np.all(cf >= 0) and np.all(cf + cf[_rev(u, v)] == cap + cap[_rev(u, v)])


def _rev(u, v):
    key = {(int(a), int(b)): i for i, (a, b) in enumerate(zip(u, v))}
    return np.array([key[(int(b), int(a))] for a, b in zip(u, v)])


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_push_pull_update_equals_dinic_and_respects_the_sides(gi):
    g = GRAPHS[gi]
    rng = np.random.default_rng(500 + gi)
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    R = oracle.Residual(g.n, g.src, g.dst, g.cap)
    R.static_init(g.s)
    R.push_relabel(g.s, g.t, 4)
    for step in range(4):
        b = W.mixed_batch(es, max(2, es.m // 10), rng, ins_cap_hi=30,
                          st_bias=(g.s, g.t, 0.3) if step % 2 else None)
        es.apply(b.u, b.v, b.cap)
        want = oracle.maxflow(g.n, *es.coo(), g.s, g.t).value
        # the sequence of R9, step by step, checking what each step promises
        side = R.cut_side()
        side[g.s], side[g.t] = 0, 1
        R.apply(g.s, b.u, b.v, b.cap)
        R.saturate_cut(side)
        u, v, cap, cf = R.slots()
        assert not np.any((side[u] == 0) & (side[v] == 1) & (cf > 0))   # no residual edge S -> T
        e1, _ = R.vertex()
        cf1 = cf.copy()
        R.push_side(g.s, g.t, side, 1, 4)
        _, _, _, cf2 = R.slots()
        e2, _ = R.vertex()
        s_slot = (side[u] == 0) & (side[v] == 0)
        assert np.array_equal(cf1[s_slot], cf2[s_slot])                  # push stays in T
        assert np.array_equal(e1[side == 0], e2[side == 0])
        R.pull_relabel(g.s, g.t, 4, side=side, want=0)
        _, _, _, cf3 = R.slots()
        e3, _ = R.vertex()
        t_slot = (side[u] == 1) & (side[v] == 1)
        assert np.array_equal(cf2[t_slot], cf3[t_slot])                  # pull stays in S
        assert np.array_equal(e2[side == 1], e3[side == 1])
        val, _, _, _ = R.push_relabel(g.s, g.t, 4)
        assert val == want


def test_push_pull_update_helper_matches_dinic_over_a_sequence():
    g = W.erdos_renyi(300, 2000, seed=77, cap_hi=100)
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    R = oracle.Residual(g.n, g.src, g.dst, g.cap)
    R.static_init(g.s)
    R.push_relabel(g.s, g.t, 8)
    rng = np.random.default_rng(78)
    for kind in ("inc", "dec", "mix", "mixed", "dec"):
        b = W.mixed_batch(es, 200, rng, ins_cap_hi=100) if kind == "mixed" else W.kind_batch(es, 200, rng, kind)
        es.apply(b.u, b.v, b.cap)
        assert R.push_pull_update(g.s, g.t, b.u, b.v, b.cap, 8) == oracle.maxflow(g.n, *es.coo(), g.s, g.t).value


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_cut_side_of_a_solved_state_is_a_minimum_cut(gi):
    # R9's S / T split, pinned to Dinic: after a solve, side 0 holds s, side 1
    # holds t, the capacity from side 0 to side 1 is the max-flow value, and
    # side 0 lies between the smallest and the largest minimum source sides
    g = GRAPHS[gi]
    R = oracle.Residual(g.n, g.src, g.dst, g.cap)
    R.static_init(g.s)
    val, *_ = R.push_relabel(g.s, g.t, 4)
    d = oracle.maxflow(g.n, g.src, g.dst, g.cap, g.s, g.t)
    assert val == d.value
    side = R.cut_side()
    assert side[g.s] == 0 and side[g.t] == 1
    u, v, cap, _ = R.slots()
    assert int(cap[(side[u] == 0) & (side[v] == 1)].sum()) == d.value
    S = side == 0
    assert np.all(S[d.smin]) and np.all(d.smax[S])
