"""Parity at full size, in the launch configuration bench.py uses.

R-MAT scale 20 (2^20 vertices, 16,085,726 merged edges): the static value and
the value after batches of 1K, 10K and 100K mixed updates equal the oracle's
Dinic value, and the downloaded state carries the max-flow/min-cut
certificate (checked on the CPU with numpy).  The 2048 x 2048 segmentation
grid: Dinic takes minutes there, so the check is the certificate plus a
feasible flow of the same value (weak duality then makes both optimal).
"""
import numpy as np
import pytest

import oracle
from paper_2511_01235_gb300 import native
from paper_2511_01235_gb300 import workloads as W
from tests.helpers import assert_certificate, flow_invariants

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rmat20():
    return W.rmat(20, 16, 0.57, 0.19, 0.19, seed=2, cap_lo=1, cap_hi=1000)


def _cert(S, value):
    su, sv, scap, scf = S.residual()
    h, e = S.vertex_state()
    return assert_certificate(S.n, S.s, S.t, su, sv, scap, scf, h, e, value)


def test_rmat20_static_and_batches(rmat20):
    g = rmat20
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    v, _, cut = S.query(cut=True)
    assert v == oracle.maxflow(g.n, g.src, g.dst, g.cap, g.s, g.t).value
    assert cut == v
    _cert(S, v)
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    rng = np.random.default_rng(77)
    for B in (1000, 10000, 100000):
        b = W.mixed_batch(es, B, rng, ins_cap_hi=1000)
        es.apply(b.u, b.v, b.cap)
        S.update(b.u, b.v, b.cap)
        v, _, cut = S.query(cut=True)
        u2, v2, c2 = es.coo()
        ref = oracle.maxflow(g.n, u2, v2, c2, g.s, g.t)
        assert v == ref.value and cut == ref.value, (B, v, cut, ref.value)
    _cert(S, v)
    S.close()


def test_rmat20_s_t_biased_batches(rmat20):
    """Batches that change the source's and sink's edges (Sec. 6.2) move the flow value."""
    g = rmat20
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    rng = np.random.default_rng(78)
    values = []
    for kind in ("inc", "dec"):
        b = W.mixed_batch(es, 2000, rng, ins_cap_hi=1000, st_bias=(g.s, g.t, 0.5),
                          frac=(1.0, 0.0, 0.0) if kind == "inc" else (0.0, 1.0, 0.0))
        es.apply(b.u, b.v, b.cap)
        S.update(b.u, b.v, b.cap)
        v = S.query()[0]
        u2, v2, c2 = es.coo()
        assert v == oracle.maxflow(g.n, u2, v2, c2, g.s, g.t).value
        values.append(v)
    S.close()


def test_grid2048_certificate_and_flow():
    G = W.GridSegmentation(side=2048, seed=3)
    g = G.graph()
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    v, _, cut = S.query(cut=True)
    assert cut == v and v > 0
    _cert(S, v)
    for k in range(2):
        b = G.window_batch(k)
        S.update(b.u, b.v, b.cap)
    v, _, cut = S.query(cut=True)
    assert cut == v
    _cert(S, v)
    u, vv, cap, f = S.get_flow()
    flow_invariants(g.n, g.s, g.t, u, vv, cap, f, v)
    S.close()


def test_rmat20_push_pull_and_pull_only(rmat20):
    # the push-pull update and the pull-only static solve at full size, against Dinic
    g = rmat20
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    rng = np.random.default_rng(78)
    for B in (10000, 100000):
        b = W.mixed_batch(es, B, rng, ins_cap_hi=1000, st_bias=(g.s, g.t, 0.3))
        es.apply(b.u, b.v, b.cap)
        S.update_pp(b.u, b.v, b.cap)
        want = oracle.maxflow(g.n, *es.coo(), g.s, g.t).value
        assert S.query()[0] == want
        _cert(S, want)
    S.resolve_static_pull()
    assert S.query()[0] == want
    _cert(S, want)
    S.close()
