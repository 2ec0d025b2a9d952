"""Push and pull on the GPU (Sec. 5.2.2, O2) against the oracle.

- The pull-relabel kernels alone (maxflow_resolve_static_pull) and the static
  push-pull give Dinic's value, and the final state is a max-flow certificate.
- The dynamic push-pull (maxflow_update_pp) gives Dinic's value after every
  batch, equal to maxflow_update's, with a certificate.
- Each of its steps keeps its promise: after step 1 no residual edge leads
  from side 0 to side 1 of the previous cut; after step 2 no overflowing
  vertex of side 1 reaches t or a deficit of side 1, and no deficit of side 0
  is reached from s or an overflowing vertex of side 0.
"""
import numpy as np
import pytest

import oracle
from paper_2511_01235_gb300 import native
from paper_2511_01235_gb300 import workloads as W

from helpers import assert_certificate

pytestmark = pytest.mark.gpu


def _families():
    G = W.GridSegmentation(side=64, seed=3, window=16, origin=(16, 16), step=1)
    return {
        "er": W.erdos_renyi(3000, 24000, seed=601, cap_hi=100),
        "rmat13": W.rmat(13, 16, 0.57, 0.19, 0.19, seed=602, cap_hi=1000),
        "grid64": G.graph(),
        "layered": W.layered_dag(5000, seed=603),
        "geometric": W.geometric(3000, seed=604),
    }


FAM = _families()


def _cert(S, g, value):
    u, v, cap, cf = S.residual()
    h, e = S.vertex_state()
    assert_certificate(g.n, g.s, g.t, u, v, cap, cf, h, e, value)


@pytest.mark.parametrize("name", list(FAM))
@pytest.mark.parametrize("cycles", [0, 1, 16])
def test_static_pull_and_static_push_pull_equal_dinic(name, cycles):
    g = FAM[name]
    want = oracle.maxflow(g.n, g.src, g.dst, g.cap, g.s, g.t).value
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t, kernel_cycles=cycles)
    S.resolve_static_pull()
    assert S.query()[0] == want
    _cert(S, g, want)
    S.resolve_static_pp()
    assert S.query()[0] == want
    _cert(S, g, want)
    S.close()


def _reach(n, u, v, cf, roots):
    import scipy.sparse as sp
    from scipy.sparse.csgraph import breadth_first_order
    m = cf > 0
    A = sp.csr_matrix((np.ones(int(m.sum()), np.int8), (u[m], v[m])), shape=(n, n))
    seen = np.zeros(n, bool)
    for r in roots:
        if not seen[r]:
            seen[breadth_first_order(A, int(r), directed=True, return_predecessors=False)] = True
    return seen


@pytest.mark.parametrize("name", ["er", "rmat13", "grid64"])
def test_push_pull_update_equals_dinic_and_update(name):
    g = FAM[name]
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    rng = np.random.default_rng(610)
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    R = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    for k in range(6):
        if name == "grid64":
            G = W.GridSegmentation(side=64, seed=3, window=16, origin=(16, 16), step=1)
            b = G.window_batch(k)
        elif k % 3 == 2:
            b = W.kind_batch(es, max(10, es.m // 50), rng, "dec")
        else:
            b = W.mixed_batch(es, max(10, es.m // 50), rng, ins_cap_hi=100,
                              st_bias=(g.s, g.t, 0.3) if k % 2 else None)
        es.apply(b.u, b.v, b.cap)
        S.update_pp(b.u, b.v, b.cap)
        R.update(b.u, b.v, b.cap)
        want = oracle.maxflow(g.n, *es.coo(), g.s, g.t).value
        assert S.query()[0] == want == R.query()[0]
        _cert(S, g, want)
    S.close()
    R.close()


@pytest.mark.parametrize("name", ["er", "rmat13"])
def test_push_pull_steps_keep_their_promises(name):
    g = FAM[name]
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    rng = np.random.default_rng(620)
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    for k in range(3):
        b = W.mixed_batch(es, max(10, es.m // 40), rng, ins_cap_hi=100, st_bias=(g.s, g.t, 0.3))
        es.apply(b.u, b.v, b.cap)
        h0, _ = S.vertex_state()
        side = (h0 < g.n).astype(np.uint8)
        side[g.s], side[g.t] = 0, 1
        C = S.clone()
        C.update_pp(b.u, b.v, b.cap, stop_after=1)
        u, v, cap, cf = C.residual()
        assert not np.any((side[u] == 0) & (side[v] == 1) & (cf > 0))
        C.close()
        C = S.clone()
        C.update_pp(b.u, b.v, b.cap, stop_after=2)
        u, v, cap, cf = C.residual()
        _, e = C.vertex_state()
        ids = np.arange(g.n)
        term = (ids == g.s) | (ids == g.t)
        # push part: from each overflowing vertex of side 1, no residual path to t or a side-1 deficit
        t_exc = ids[(side == 1) & (e > 0) & ~term]
        t_sink = ((side == 1) & (e < 0) & ~term) | (ids == g.t)
        if t_exc.size:
            assert not np.any(_reach(g.n, u, v, cf, t_exc) & t_sink)
        # pull part: no side-0 deficit is reached from s or a side-0 overflowing vertex
        s_src = list(ids[(side == 0) & (e > 0) & ~term]) + [g.s]
        s_def = (side == 0) & (e < 0) & ~term
        assert not np.any(_reach(g.n, u, v, cf, s_src) & s_def)
        # finishing from there gives the max flow
        C.resolve()
        want = oracle.maxflow(g.n, *es.coo(), g.s, g.t).value
        assert C.query()[0] == want
        C.close()
        S.update_pp(b.u, b.v, b.cap)
        assert S.query()[0] == want
    S.close()


def test_push_pull_after_an_unsolved_state_falls_back_to_update():
    g = FAM["er"]
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    rng = np.random.default_rng(630)
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    b = W.mixed_batch(es, 200, rng, ins_cap_hi=100)
    es.apply(b.u, b.v, b.cap)
    S.apply(b.u, b.v, b.cap)                    # unsolved now
    b2 = W.mixed_batch(es, 200, rng, ins_cap_hi=100)
    es.apply(b2.u, b2.v, b2.cap)
    S.update_pp(b2.u, b2.v, b2.cap)
    assert S.query()[0] == oracle.maxflow(g.n, *es.coo(), g.s, g.t).value
    assert native.load().maxflow_update_pp(S.h, None, 0) == native.ERR_INVALID      # no batch
    with pytest.raises(native.MaxflowError) as ei:
        S.update_pp(b2.u, b2.v, b2.cap, stop_after=7)
    assert ei.value.code == native.ERR_INVALID
    assert S.query()[0] == oracle.maxflow(g.n, *es.coo(), g.s, g.t).value   # unchanged by the refusals
    S.close()


def _tiny(n, edges, s, t):
    src = np.array([e[0] for e in edges], np.int32)
    dst = np.array([e[1] for e in edges], np.int32)
    cap = np.array([e[2] for e in edges], np.int32)
    return src, dst, cap


@pytest.mark.parametrize("case", ["no_path", "direct_st", "isolated", "chain"])
def test_push_pull_degenerate_graphs(case):
    if case == "no_path":                    # s reaches nothing that reaches t: value 0
        n, edges = 6, [(0, 1, 5), (1, 2, 5), (3, 5, 7), (4, 3, 2)]
    elif case == "direct_st":                # the only path is the edge s -> t
        n, edges = 4, [(0, 3, 9), (1, 2, 4)]
    elif case == "isolated":                 # s and t without edges
        n, edges = 5, [(1, 2, 3), (2, 3, 3)]
    else:                                    # a path whose middle edge is the cut
        n, edges = 5, [(0, 1, 10), (1, 2, 3), (2, 3, 10), (3, 4, 10)]
    s, t = 0, n - 1
    src, dst, cap = _tiny(n, edges, s, t)
    want = oracle.maxflow(n, src, dst, cap, s, t).value
    S = native.Solver(n, src, dst, cap, s, t)
    for fn in ("resolve_static_pull", "resolve_static_pp"):
        getattr(S, fn)()
        assert S.query()[0] == want, fn
    # an empty batch, then a batch that opens (or closes) a path, both by push-pull
    z = np.zeros(0, np.int32)
    S.update_pp(z, z, z)
    assert S.query()[0] == want
    es = W.EdgeSet(n, src, dst, cap)
    bu, bv, bc = np.array([s, 1], np.int32), np.array([1, t], np.int32), np.array([4, 6], np.int32)
    es.apply(bu, bv, bc)
    S.update_pp(bu, bv, bc)
    assert S.query()[0] == oracle.maxflow(n, *es.coo(), s, t).value
    S.close()
