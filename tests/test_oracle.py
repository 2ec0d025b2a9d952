"""Pins for the CPU oracle (no GPU).

Each check ties the oracle to something other than itself: brute-force
enumeration of every s-t cut, scipy's own max-flow routines, an independent
Edmonds-Karp, closed forms, flow invariants, scipy shortest paths, and
hand-derived fixtures under tests/golden/.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import oracle
from paper_2511_01235_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute_min_cuts(n, src, dst, cap, s, t):
    """Every s-t cut: returns (min capacity, intersection and union of all minimum source sides)."""
    others = [x for x in range(n) if x not in (s, t)]
    best, sides = None, []
    for bits in range(1 << len(others)):
        S = np.zeros(n, bool)
        S[s] = True
        for i, x in enumerate(others):
            if bits >> i & 1:
                S[x] = True
        c = int(sum(int(c) for u, v, c in zip(src, dst, cap) if S[u] and not S[v]))
        if best is None or c < best:
            best, sides = c, [S]
        elif c == best:
            sides.append(S)
    inter = np.logical_and.reduce(sides)
    union = np.logical_or.reduce(sides)
    return best, inter, union


@pytest.mark.parametrize("seed", range(120))
def test_dinic_equals_bruteforce_min_cut(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 10))
    m = int(rng.integers(0, 3 * n + 1))
    src, dst, cap = W.random_multigraph(n, m, seed=seed, cap_hi=9)
    s, t = 0, n - 1
    best, inter, union = brute_min_cuts(n, src, dst, cap, s, t)
    r = oracle.maxflow(n, src, dst, cap, s, t)
    assert r.value == best
    assert r.cut_cap == best
    np.testing.assert_array_equal(r.smin, inter)
    np.testing.assert_array_equal(r.smax, union)


def _scipy_value(n, src, dst, cap, s, t, method):
    keep = src != dst
    g = sp.csr_matrix((cap[keep].astype(np.int32), (src[keep], dst[keep])), shape=(n, n))
    g.sum_duplicates()
    return int(csg.maximum_flow(g, s, t, method=method).flow_value)


@pytest.mark.parametrize("seed", range(30))
def test_dinic_equals_scipy(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(20, 400))
    m = int(rng.integers(n, 8 * n))
    src, dst, cap = W.random_multigraph(n, m, seed=1000 + seed, cap_hi=100)
    s, t = int(rng.integers(0, n)), int(rng.integers(0, n))
    if s == t:
        t = (s + 1) % n
    v = oracle.maxflow(n, src, dst, cap, s, t).value
    assert v == _scipy_value(n, src, dst, cap, s, t, "dinic")
    assert v == _scipy_value(n, src, dst, cap, s, t, "edmonds_karp")


def test_dinic_equals_scipy_er_small():
    g = W.er_small()
    v = oracle.maxflow(g.n, g.src, g.dst, g.cap, g.s, g.t).value
    assert v == _scipy_value(g.n, g.src, g.dst, g.cap, g.s, g.t, "dinic")


@pytest.mark.parametrize("seed", range(40))
def test_dinic_equals_edmonds_karp(seed):
    rng = np.random.default_rng(2000 + seed)
    n = int(rng.integers(2, 60))
    m = int(rng.integers(0, 6 * n))
    src, dst, cap = W.random_multigraph(n, m, seed=2000 + seed, cap_hi=50)
    assert oracle.maxflow(n, src, dst, cap, 0, n - 1).value == oracle.maxflow_ek(n, src, dst, cap, 0, n - 1)


def check_flow_invariants(n, src, dst, cap, s, t, flow, value):
    src, dst, cap, flow = (np.asarray(a, np.int64) for a in (src, dst, cap, flow))
    assert np.all(flow >= 0) and np.all(flow <= cap)
    inflow = np.bincount(dst, weights=flow, minlength=n).astype(np.int64)
    outflow = np.bincount(src, weights=flow, minlength=n).astype(np.int64)
    net = inflow - outflow
    mask = np.ones(n, bool)
    mask[[s, t]] = False
    assert np.all(net[mask] == 0)
    assert -net[s] == value and net[t] == value


@pytest.mark.parametrize("seed", range(25))
def test_dinic_flow_invariants(seed):
    rng = np.random.default_rng(3000 + seed)
    n = int(rng.integers(2, 300))
    src, dst, cap = W.random_multigraph(n, int(rng.integers(0, 6 * n)), seed=3000 + seed, cap_hi=30)
    r = oracle.maxflow(n, src, dst, cap, 0, n - 1)
    check_flow_invariants(n, src, dst, cap, 0, n - 1, r.flow, r.value)
    assert r.cut_cap == r.value
    assert np.all(r.smin <= r.smax) and r.smin[0] and not r.smax[n - 1]


# --- closed forms -------------------------------------------------------------


def test_closed_form_path():
    caps = [7, 3, 9, 4, 11]
    n = len(caps) + 1
    assert oracle.maxflow(n, range(n - 1), range(1, n), caps, 0, n - 1).value == 3


def test_closed_form_disjoint_paths():
    rng = np.random.default_rng(5)
    src, dst, cap, total, nxt = [], [], [], 0, 2
    for _ in range(6):
        L = int(rng.integers(1, 5))
        cs = rng.integers(1, 50, size=L + 1)
        path = [0] + list(range(nxt, nxt + L)) + [1]
        nxt += L
        for (a, b), c in zip(zip(path[:-1], path[1:]), cs):
            src.append(a); dst.append(b); cap.append(int(c))
        total += int(cs.min())
    assert oracle.maxflow(nxt, src, dst, cap, 0, 1).value == total


@pytest.mark.parametrize("a,b", [(1, 1), (3, 5), (7, 2), (6, 6)])
def test_closed_form_bipartite(a, b):
    n = a + b + 2
    s, t = 0, n - 1
    src, dst = [], []
    for i in range(a):
        src.append(s); dst.append(1 + i)
        for j in range(b):
            src.append(1 + i); dst.append(1 + a + j)
    for j in range(b):
        src.append(1 + a + j); dst.append(t)
    assert oracle.maxflow(n, src, dst, [1] * len(src), s, t).value == min(a, b)


def test_closed_form_disconnected_and_zero():
    assert oracle.maxflow(4, [0, 2], [1, 3], [5, 5], 0, 3).value == 0
    assert oracle.maxflow(3, [0, 1], [1, 2], [0, 0], 0, 2).value == 0
    assert oracle.maxflow(2, [], [], [], 0, 1).value == 0


@pytest.mark.parametrize("seed", range(10))
def test_closed_form_scaling(seed):
    src, dst, cap = W.random_multigraph(40, 200, seed=seed, cap_hi=20)
    v1 = oracle.maxflow(40, src, dst, cap, 0, 39).value
    assert oracle.maxflow(40, src, dst, 2 * cap, 0, 39).value == 2 * v1


def test_closed_form_layered_known_cut():
    # two layers joined only by a middle edge set of known total; everything else huge
    rng = np.random.default_rng(9)
    k = 12
    A = list(range(1, k + 1))
    B = list(range(k + 1, 2 * k + 1))
    s, t = 0, 2 * k + 1
    src, dst, cap = [], [], []
    big = 10 ** 6
    for x in A:
        src.append(s); dst.append(x); cap.append(big)
        for y in A:
            if x != y:
                src.append(x); dst.append(y); cap.append(big)
    for y in B:
        src.append(y); dst.append(t); cap.append(big)
    mid = 0
    for _ in range(30):
        x, y = int(rng.choice(A)), int(rng.choice(B))
        c = int(rng.integers(1, 100))
        src.append(x); dst.append(y); cap.append(c)
        mid += c
    assert oracle.maxflow(2 * k + 2, src, dst, cap, s, t).value == mid


def test_merge_sums_parallel_drops_loops():
    u, v, c = oracle.merge(4, [0, 0, 1, 2, 2, 0], [1, 1, 1, 3, 3, 2], [2, 5, 7, 1, 1, 0])
    assert list(zip(u, v, c)) == [(0, 1, 7), (0, 2, 0), (2, 3, 2)]


# --- residual state, heights, apply -----------------------------------------------


def _slots_dict(R):
    u, v, cap, cf = R.slots()
    return {(int(a), int(b)): (int(c), int(d)) for a, b, c, d in zip(u, v, cap, cf)}


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _edges(fx):
    E = np.array(fx["edges"], dtype=np.int64).reshape(-1, 3)
    return E[:, 0], E[:, 1], E[:, 2]


def test_golden_static_init_heights():
    fx = _load("static_init_heights.json")
    src, dst, cap = _edges(fx)
    R = oracle.Residual(fx["n"], src, dst, cap)
    R.static_init(fx["s"])
    assert _slots_dict(R) == {(a, b): (c, d) for a, b, c, d in fx["after_init"]["slots"]}
    e, _ = R.vertex()
    assert list(e) == fx["after_init"]["excess"]
    assert list(R.heights(fx["s"], fx["t"])) == fx["heights"]
    v, *_ = R.push_relabel(fx["s"], fx["t"], kernel_cycles=2)
    assert v == fx["value"]


@pytest.mark.parametrize("name", ["apply_decrease_below_flow.json", "apply_source_edge_deficit.json",
                                  "apply_insert_and_resaturate.json"])
def test_golden_apply(name):
    fx = _load(name)
    src, dst, cap = _edges(fx)
    R = oracle.Residual(fx["n"], src, dst, cap)
    F = np.array(fx["flow"]).reshape(-1, 3)
    R.set_flow(F[:, 0], F[:, 1], F[:, 2])
    Bt = np.array(fx["batch"]).reshape(-1, 3)
    R.apply(fx["s"], Bt[:, 0], Bt[:, 1], Bt[:, 2])
    assert _slots_dict(R) == {(a, b): (c, d) for a, b, c, d in fx["after_apply"]["slots"]}
    e, _ = R.vertex()
    assert list(e) == fx["after_apply"]["excess"]
    if "heights_after_apply" in fx:
        assert list(R.heights(fx["s"], fx["t"])) == fx["heights_after_apply"]
    v, *_ = R.push_relabel(fx["s"], fx["t"], kernel_cycles=3)
    assert v == fx["value"]
    # and the plain definition agrees
    es = W.EdgeSet(fx["n"], src, dst, cap)
    es.apply(Bt[:, 0], Bt[:, 1], Bt[:, 2])
    u2, v2, c2 = es.coo()
    assert oracle.maxflow(fx["n"], u2, v2, c2, fx["s"], fx["t"]).value == fx["value"]


def _random_flow(rng, u, v, c, frac=0.6):
    f = np.where(rng.random(c.size) < frac, np.floor(rng.random(c.size) * (c + 1)), 0).astype(np.int32)
    return np.minimum(f, c).astype(np.int32)


@pytest.mark.parametrize("seed", range(20))
def test_excess_matches_in_minus_out(seed):
    rng = np.random.default_rng(4000 + seed)
    n = int(rng.integers(3, 200))
    src, dst, cap = W.random_multigraph(n, 5 * n, seed=4000 + seed, cap_hi=30)
    u, v, c = oracle.merge(n, src, dst, cap)
    f = _random_flow(rng, u, v, c)
    R = oracle.Residual(n, src, dst, cap)
    R.set_flow(u, v, f)
    e, _ = R.vertex()
    ref = np.bincount(v, weights=f, minlength=n) - np.bincount(u, weights=f, minlength=n)
    np.testing.assert_array_equal(e, ref.astype(np.int64))
    # pair-sum invariant (Sec. 3.1, Theorem 3.3)
    S = _slots_dict(R)
    for (a, b), (ca, fa) in S.items():
        cb, fb = S[(b, a)]
        assert fa + fb == ca + cb and fa >= 0


@pytest.mark.parametrize("seed", range(20))
def test_heights_equal_scipy_shortest_paths(seed):
    rng = np.random.default_rng(5000 + seed)
    n = int(rng.integers(3, 300))
    src, dst, cap = W.random_multigraph(n, 4 * n, seed=5000 + seed, cap_hi=10, zero_frac=0.3)
    s, t = 0, n - 1
    u, v, c = oracle.merge(n, src, dst, cap)
    f = _random_flow(rng, u, v, c)
    R = oracle.Residual(n, src, dst, cap)
    R.set_flow(u, v, f)
    e, _ = R.vertex()
    h = R.heights(s, t, deficit_roots=True)
    su, sv, scap, scf = R.slots()
    # residual edge (x, y) with c_f > 0, s removed; distances from x to the root set
    keep = (scf > 0) & (su != s) & (sv != s)
    roots = [t] + [x for x in range(n) if x not in (s, t) and e[x] < 0]
    G = sp.csr_matrix((np.ones(int(keep.sum())), (sv[keep], su[keep])), shape=(n, n))  # reversed
    D = csg.shortest_path(G, unweighted=True, directed=True, indices=roots)
    d = D.min(axis=0)
    ref = np.where(np.isinf(d), n, d).astype(np.int64)
    ref[s] = n
    np.testing.assert_array_equal(h, ref)
    # static BFS: only t is a root
    h2 = R.heights(s, t, deficit_roots=False)
    D2 = csg.shortest_path(G, unweighted=True, directed=True, indices=[t])[0]
    ref2 = np.where(np.isinf(D2), n, D2).astype(np.int64)
    ref2[s] = n
    np.testing.assert_array_equal(h2, ref2)


@pytest.mark.parametrize("seed", range(40))
def test_sequential_static_push_relabel_equals_dinic(seed):
    rng = np.random.default_rng(6000 + seed)
    n = int(rng.integers(2, 150))
    src, dst, cap = W.random_multigraph(n, int(rng.integers(0, 8 * n)), seed=6000 + seed, cap_hi=40)
    s, t = 0, n - 1
    R = oracle.Residual(n, src, dst, cap)
    R.static_init(s)
    v, it, pushes, relabels = R.push_relabel(s, t, kernel_cycles=int(rng.integers(1, 9)))
    assert v == oracle.maxflow(n, src, dst, cap, s, t).value
    cut, bad = R.cut()
    assert bad == 0 and cut == v        # Theorem 3.4 certificate


@pytest.mark.parametrize("seed", range(25))
def test_sequential_dynamic_push_relabel_equals_dinic(seed):
    rng = np.random.default_rng(7000 + seed)
    n = int(rng.integers(4, 200))
    g = W.erdos_renyi(n, min(4 * n, n * (n - 1) // 2), seed=7000 + seed, cap_hi=60)
    R = oracle.Residual(n, g.src, g.dst, g.cap)
    R.static_init(g.s)
    R.push_relabel(g.s, g.t, 4)
    es = W.EdgeSet(n, g.src, g.dst, g.cap)
    for b in range(4):
        B = int(rng.integers(1, max(2, es.m // 3)))
        bt = W.mixed_batch(es, B, rng, ins_cap_hi=60)
        es.apply(bt.u, bt.v, bt.cap)
        R.apply(g.s, bt.u, bt.v, bt.cap)
        v, *_ = R.push_relabel(g.s, g.t, int(rng.integers(1, 6)))
        u2, v2, c2 = es.coo()
        assert v == oracle.maxflow(n, u2, v2, c2, g.s, g.t).value
        cut, bad = R.cut()
        assert bad == 0 and cut == v


@pytest.mark.parametrize("seed", range(20))
def test_dynamic_from_arbitrary_pseudoflow(seed):
    """Alg. 5 from any flow assignment 0 <= f <= c reaches the max flow (Sec. 4.3)."""
    rng = np.random.default_rng(8000 + seed)
    n = int(rng.integers(3, 150))
    src, dst, cap = W.random_multigraph(n, 5 * n, seed=8000 + seed, cap_hi=25)
    u, v, c = oracle.merge(n, src, dst, cap)
    f = _random_flow(rng, u, v, c, frac=0.8)
    R = oracle.Residual(n, src, dst, cap)
    R.set_flow(u, v, f)
    R.apply(0, [], [], [])
    val, *_ = R.push_relabel(0, n - 1, 3)
    assert val == oracle.maxflow(n, src, dst, cap, 0, n - 1).value


def test_apply_rejects_invalid_batch_unchanged():
    R = oracle.Residual(3, [0, 1], [1, 2], [5, 5])
    before = _slots_dict(R)
    with pytest.raises(ValueError):
        R.apply(0, [0, 1], [1, 7], [3, 3])
    with pytest.raises(ValueError):
        R.apply(0, [0], [1], [-1])
    assert _slots_dict(R) == before


def test_apply_last_update_wins_and_loops_ignored():
    R = oracle.Residual(3, [0, 1], [1, 2], [5, 5])
    R.apply(0, [1, 1, 2, 1], [2, 2, 2, 2], [9, 1, 4, 3])
    S = _slots_dict(R)
    assert S[(1, 2)][0] == 3 and (2, 2) not in S


def _brute_min_cuts_vectorised(n, src, dst, cap, s, t):
    """Every s-t cut at once (numpy): (min capacity, intersection and union of all minimum source sides)."""
    others = np.array([x for x in range(n) if x not in (s, t)], np.int64)
    k = others.size
    codes = np.arange(1 << k, dtype=np.int64)
    S = np.zeros((codes.size, n), bool)
    S[:, s] = True
    S[:, others] = ((codes[:, None] >> np.arange(k)) & 1).astype(bool)
    keep = src != dst
    u, v, c = src[keep], dst[keep], cap[keep].astype(np.int64)
    caps = (S[:, u] & ~S[:, v]).astype(np.int64) @ c
    best = int(caps.min())
    sides = S[caps == best]
    return best, sides.all(axis=0), sides.any(axis=0)


@pytest.mark.parametrize("seed", range(12))
def test_dinic_equals_bruteforce_min_cut_up_to_18_vertices(seed):
    # every s-t cut of graphs of 12-18 vertices (up to 2^16 cuts each)
    rng = np.random.default_rng(5000 + seed)
    n = int(rng.integers(12, 19))
    m = int(rng.integers(n, 4 * n))
    src, dst, cap = W.random_multigraph(n, m, seed=5000 + seed, cap_hi=9)
    s, t = 0, n - 1
    best, inter, union = _brute_min_cuts_vectorised(n, src, dst, cap, s, t)
    r = oracle.maxflow(n, src, dst, cap, s, t)
    assert r.value == best == r.cut_cap
    np.testing.assert_array_equal(r.smin, inter)
    np.testing.assert_array_equal(r.smax, union)


def test_vectorised_enumeration_agrees_with_the_loop():
    for seed in range(20):
        rng = np.random.default_rng(6000 + seed)
        n = int(rng.integers(2, 9))
        src, dst, cap = W.random_multigraph(n, int(rng.integers(0, 3 * n + 1)), seed=6000 + seed, cap_hi=9)
        a = brute_min_cuts(n, src, dst, cap, 0, n - 1)
        b = _brute_min_cuts_vectorised(n, src, dst, cap, 0, n - 1)
        assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_dinic_equals_edmonds_karp_on_ten_thousand_graphs():
    # the two independent algorithms agree on 10,000 random small and medium multigraphs
    rng = np.random.default_rng(7000)
    for i in range(10_000):
        n = int(rng.integers(2, 40))
        m = int(rng.integers(0, 5 * n))
        src = rng.integers(0, n, m).astype(np.int32)
        dst = rng.integers(0, n, m).astype(np.int32)
        cap = rng.integers(0, 30, m).astype(np.int32)
        s, t = (0, n - 1) if i % 2 else tuple(int(x) for x in rng.choice(n, 2, replace=False))
        assert oracle.maxflow(n, src, dst, cap, s, t).value == oracle.maxflow_ek(n, src, dst, cap, s, t), i
