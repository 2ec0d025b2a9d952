"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer work, so every compared quantity is exact: the flow value and the
min-cut capacity equal the oracle's Dinic result bit for bit; the cut side A
lies between the oracle's S_min and S_max (every minimum cut does, and
several may exist); heights of a backward BFS equal the oracle's BFS
distances; the residual state after a batch repair equals the oracle's
restatement of Alg. 5 slot by slot.  Flows are not unique, so extracted flows
are checked for capacity, conservation and value.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2511_01235_gb300 import native
from paper_2511_01235_gb300 import workloads as W
from tests.helpers import assert_certificate, flow_invariants, slot_dict

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    native.load()
    yield
    torch.cuda.synchronize()


def check_against_oracle(S, n, src, dst, cap, s, t):
    ref = oracle.maxflow(n, src, dst, cap, s, t)
    v, side, cut = S.query(side=True, cut=True)
    assert v == ref.value, (v, ref.value)
    assert cut == ref.value, (cut, ref.value)
    assert np.all(ref.smin <= side) and np.all(side <= ref.smax)
    chk = S.check()
    assert chk["pair_violations"] == 0 and chk["excess_mismatch"] == 0, chk
    assert chk["residual_cross_edges"] == 0 and chk["active"] == 0, chk
    assert chk["cut_cap"] == v and chk["value"] == v, chk
    return v


def cpu_certificate(S, value):
    su, sv, scap, scf = S.residual()
    h, e = S.vertex_state()
    return assert_certificate(S.n, S.s, S.t, su, sv, scap, scf, h, e, value)


# ---------------------------------------------------------------------------
# static solve
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("seed", range(24))
def test_static_random_multigraphs(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 400))
    m = int(rng.integers(0, 8 * n + 1))
    src, dst, cap = W.random_multigraph(n, m, seed=100 + seed, cap_hi=int(rng.integers(1, 1000)))
    s = int(rng.integers(0, n))
    t = int((s + 1 + rng.integers(0, n - 1)) % n)
    S = native.Solver(n, src, dst, cap, s, t, kernel_cycles=int(rng.integers(0, 9)))
    v = check_against_oracle(S, n, src, dst, cap, s, t)
    cpu_certificate(S, v)
    S.close()


@pytest.mark.parametrize("grid", [1, 2, 7, 0])
def test_static_grid_sizes(grid):
    g = W.erdos_renyi(3000, 24000, seed=9, cap_hi=100)
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t, grid_blocks=grid)
    check_against_oracle(S, g.n, g.src, g.dst, g.cap, g.s, g.t)
    S.close()


def test_static_hub_rows():
    """Rows above the hub threshold (4096 slots) take the CTA / grid-wide paths."""
    rng = np.random.default_rng(3)
    n = 20000
    hubs = [0, 1, 2]
    src, dst = [], []
    for hb in hubs:
        others = rng.choice(np.arange(3, n), size=6000, replace=False)
        src += [hb] * 3000 + list(others[3000:])
        dst += list(others[:3000]) + [hb] * 3000
    src += list(rng.integers(3, n, size=60000))
    dst += list(rng.integers(3, n, size=60000))
    cap = rng.integers(1, 50, size=len(src))
    for s, t in [(0, 1), (5, 2), (1, 7)]:
        S = native.Solver(n, src, dst, cap, s, t)
        v = check_against_oracle(S, n, np.array(src), np.array(dst), cap, s, t)
        cpu_certificate(S, v)
        S.close()


def test_static_multigraph_semantics():
    # parallel edges summed, self-loops dropped, zero capacities kept
    src = [0, 0, 1, 1, 2, 2, 0]
    dst = [1, 1, 1, 3, 3, 3, 2]
    cap = [2, 3, 9, 4, 1, 1, 0]
    S = native.Solver(4, src, dst, cap, 0, 3)
    assert S.query()[0] == 4
    S.close()


def test_static_no_path_and_trivial():
    S = native.Solver(4, [0, 2], [1, 3], [5, 5], 0, 3)
    assert S.query(cut=True)[0::2] == (0, 0)
    S.close()
    S = native.Solver(2, [], [], [], 0, 1)
    assert S.query()[0] == 0
    S.close()
    S = native.Solver(2, [0, 1], [1, 0], [7, 3], 0, 1)
    assert S.query()[0] == 7
    S.close()


@pytest.mark.parametrize("topo,fix", [(False, True), (True, False), (False, False)])
def test_static_ablations(topo, fix):
    g = W.erdos_renyi(2000, 16000, seed=21, cap_hi=100)
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t, data_driven=not topo, fix_steep=fix)
    check_against_oracle(S, g.n, g.src, g.dst, g.cap, g.s, g.t)
    S.close()


# ---------------------------------------------------------------------------
# incremental re-solve
# ---------------------------------------------------------------------------


def run_dynamic(g, batches_fn, nb, **kw):
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t, **kw)
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    check_against_oracle(S, g.n, g.src, g.dst, g.cap, g.s, g.t)
    for k in range(nb):
        b = batches_fn(es, k)
        es.apply(b.u, b.v, b.cap)
        S.update(b.u, b.v, b.cap)
        u2, v2, c2 = es.coo()
        check_against_oracle(S, g.n, u2, v2, c2, g.s, g.t)
    return S, es


def test_er_small_ten_batches():
    """Erdos-Renyi n=4096, m=32768, caps U[1,100]; static solve, then 10 mixed batches of 256."""
    g = W.er_small()
    rng = np.random.default_rng(11)
    S, es = run_dynamic(g, lambda es, k: W.mixed_batch(es, 256, rng, ins_cap_hi=100), 10)
    v = S.query()[0]
    cpu_certificate(S, v)
    u, vv, cap, f = S.get_flow()
    flow_invariants(g.n, g.s, g.t, u, vv, cap, f, v)
    S.close()


@pytest.mark.parametrize("kind", ["inc", "dec", "mix"])
def test_paper_shaped_batches(kind):
    """Increase-only, decrease-only and half/half batches (Sec. 6.2.1-6.2.3), biased to s/t edges."""
    g = W.erdos_renyi(3000, 24000, seed=31, cap_hi=100)
    rng = np.random.default_rng(32)
    run_dynamic(g, lambda es, k: W.kind_batch(es, 300, rng, kind), 6)[0].close()


@pytest.mark.parametrize("seed", range(12))
def test_random_dynamic(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(4, 600))
    g = W.erdos_renyi(n, min(6 * n, n * (n - 1) // 2), seed=500 + seed, cap_hi=int(rng.integers(1, 1000)))

    def mk(es, k):
        B = int(rng.integers(1, max(2, es.m // 4)))
        bias = (g.s, g.t, 0.3) if k % 2 else None
        return W.mixed_batch(es, B, rng, ins_cap_hi=100, st_bias=bias)

    # odd seeds run remove-invalid-edges (Alg. 3) after every discharge, even ones not (the default)
    S, _ = run_dynamic(g, mk, 5, kernel_cycles=int(rng.integers(0, 6)), fix_steep=bool(seed % 2))
    S.close()


def test_device_batches_match_host():
    import torch
    g = W.erdos_renyi(2000, 16000, seed=41, cap_hi=100)
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    rng = np.random.default_rng(42)
    A = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    B = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    for _ in range(4):
        b = W.mixed_batch(es, 200, rng, ins_cap_hi=100)
        es.apply(b.u, b.v, b.cap)
        A.update(b.u, b.v, b.cap)
        B.update(torch.from_numpy(b.u).cuda(), torch.from_numpy(b.v).cuda(), torch.from_numpy(b.cap).cuda())
        assert A.query()[0] == B.query()[0]
    u2, v2, c2 = es.coo()
    check_against_oracle(B, g.n, u2, v2, c2, g.s, g.t)
    A.close()
    B.close()


def test_duplicates_selfloops_and_empty_batch():
    g = W.erdos_renyi(500, 3000, seed=51, cap_hi=50)
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    u = np.array([g.src[0], g.src[0], 7, 7, g.s, 3, 3], np.int32)
    v = np.array([g.dst[0], g.dst[0], 7, 9, 11, 4, 4], np.int32)
    c = np.array([90, 1, 5, 40, 60, 0, 33], np.int32)
    es.apply(u, v, c)
    S.update(u, v, c)
    u2, v2, c2 = es.coo()
    check_against_oracle(S, g.n, u2, v2, c2, g.s, g.t)
    S.update(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32))
    check_against_oracle(S, g.n, u2, v2, c2, g.s, g.t)
    S.close()


def test_resolve_static_matches_incremental():
    g = W.erdos_renyi(3000, 20000, seed=61, cap_hi=100)
    rng = np.random.default_rng(62)
    S, es = run_dynamic(g, lambda es, k: W.mixed_batch(es, 500, rng, ins_cap_hi=100), 3)
    v_inc = S.query()[0]
    S.resolve_static()
    u2, v2, c2 = es.coo()
    assert check_against_oracle(S, g.n, u2, v2, c2, g.s, g.t) == v_inc
    S.close()


def test_slack_overflow_rebuild():
    """Insertions into rows without spare slots rebuild the layout and keep the flow."""
    g = W.erdos_renyi(800, 4000, seed=71, cap_hi=100)
    rng = np.random.default_rng(72)
    S, es = run_dynamic(g, lambda es, k: W.mixed_batch(es, 400, rng, ins_cap_hi=100, frac=(0.2, 0.2, 0.5)), 4,
                        slack_factor=0.0, slack_min=0)
    assert S.stats()["rebuilds"] >= 1
    S.close()


def test_kernel_launch_counter():
    """maxflow_kernel_launches: an update is one launch; an update whose insertion
    overflows a row's slack adds the rebuild's seven kernels (row sizes, a
    three-pass scan, the pieces of long rows, the row copy, the demand reset)
    and a second solve."""
    g = W.erdos_renyi(800, 4000, seed=73, cap_hi=100)
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t, slack_factor=0.0, slack_min=0)
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    rng = np.random.default_rng(74)
    b = W.kind_batch(es, 50, rng, "inc")                 # existing edges only: no insertion
    es.apply(b.u, b.v, b.cap)
    l0, r0 = native.kernel_launches(), S.stats()["rebuilds"]
    S.update(b.u, b.v, b.cap)
    assert native.kernel_launches() - l0 == 1 and S.stats()["rebuilds"] == r0
    # rows hold a multiple of 4 slots; with no slack a row is full exactly when its
    # vertex has a multiple of 4 neighbours (in either direction)
    nb = np.zeros(g.n, np.int64)
    pairs = set()
    for a, c in zip(es.keys // g.n, es.keys % g.n):
        pairs.add((min(int(a), int(c)), max(int(a), int(c))))
    for a, c in pairs:
        nb[a] += 1
        nb[c] += 1
    u, v = next((a, c) for a in range(1, g.n) if nb[a] % 4 == 0 for c in range(1, g.n)
                if nb[c] % 4 == 0 and a != c and not es.contains(a, c) and not es.contains(c, a) and g.t not in (a, c))
    bu, bv, bc = np.array([u], np.int32), np.array([v], np.int32), np.array([7], np.int32)
    es.apply(bu, bv, bc)
    l0 = native.kernel_launches()
    S.update(bu, bv, bc)                                 # a new pair: both rows are full
    assert S.stats()["rebuilds"] == r0 + 1
    assert native.kernel_launches() - l0 == 9
    u2, v2, c2 = es.coo()
    check_against_oracle(S, g.n, u2, v2, c2, g.s, g.t)
    S.close()


# ---------------------------------------------------------------------------
# step-level parity: heights (Alg. 4/6) and batch repair (Alg. 5)
# ---------------------------------------------------------------------------


def _random_flow(rng, c, frac=0.7):
    f = np.where(rng.random(c.size) < frac, np.floor(rng.random(c.size) * (c + 1)), 0)
    return np.minimum(f, c).astype(np.int32)


@pytest.mark.parametrize("seed", range(10))
def test_bfs_heights_exact(seed):
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(3, 3000))
    src, dst, cap = W.random_multigraph(n, 5 * n, seed=700 + seed, cap_hi=20, zero_frac=0.3)
    s, t = 0, n - 1
    mu, mv, mc = oracle.merge(n, src, dst, cap)
    f = _random_flow(rng, mc)
    R = oracle.Residual(n, src, dst, cap)
    R.set_flow(mu, mv, f)
    want = R.heights(s, t, deficit_roots=True)
    S = native.Solver(n, src, dst, cap, s, t)
    S.set_flow(mu, mv, f)
    S.global_relabel()
    h, e = S.vertex_state()
    want_e, _ = R.vertex()
    np.testing.assert_array_equal(e, want_e)
    np.testing.assert_array_equal(h, want)
    S.close()


def test_bfs_heights_static_init_state():
    g = W.erdos_renyi(4096, 32768, seed=1, cap_hi=100)
    R = oracle.Residual(g.n, g.src, g.dst, g.cap)
    R.static_init(g.s)
    want = R.heights(g.s, g.t, deficit_roots=True)
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    out = g.src == g.s
    S.set_flow(g.src[out], g.dst[out], g.cap[out])
    S.global_relabel()
    h, _ = S.vertex_state()
    np.testing.assert_array_equal(h, want)
    S.close()


@pytest.mark.parametrize("seed", range(10))
def test_apply_exact(seed):
    rng = np.random.default_rng(800 + seed)
    n = int(rng.integers(4, 2000))
    g = W.erdos_renyi(n, min(5 * n, n * (n - 1) // 2), seed=800 + seed, cap_hi=60)
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    mu, mv, mc = oracle.merge(n, g.src, g.dst, g.cap)
    f = _random_flow(rng, mc)
    R = oracle.Residual(n, g.src, g.dst, g.cap)
    R.set_flow(mu, mv, f)
    S = native.Solver(n, g.src, g.dst, g.cap, g.s, g.t)
    S.set_flow(mu, mv, f)
    B = int(rng.integers(1, max(2, es.m // 2)))
    b = W.mixed_batch(es, B, rng, ins_cap_hi=60, st_bias=(g.s, g.t, 0.3))
    # duplicates of a pair in the batch: last wins
    u = np.concatenate([b.u, b.u[:5]])
    v = np.concatenate([b.v, b.v[:5]])
    c = np.concatenate([b.cap, (b.cap[:5] + 3)]).astype(np.int32)
    R.apply(g.s, u, v, c)
    S.apply(u, v, c)
    assert slot_dict(*S.residual()) == slot_dict(*R.slots())
    _, e = S.vertex_state()
    want_e, _ = R.vertex()
    np.testing.assert_array_equal(e, want_e)
    S.close()


@pytest.mark.parametrize("name", ["apply_decrease_below_flow.json", "apply_source_edge_deficit.json",
                                  "apply_insert_and_resaturate.json"])
def test_golden_apply_gpu(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        fx = json.load(fh)
    E = np.array(fx["edges"]).reshape(-1, 3)
    F = np.array(fx["flow"]).reshape(-1, 3)
    Bt = np.array(fx["batch"]).reshape(-1, 3)
    S = native.Solver(fx["n"], E[:, 0], E[:, 1], E[:, 2], fx["s"], fx["t"])
    S.set_flow(F[:, 0], F[:, 1], F[:, 2])
    S.apply(Bt[:, 0], Bt[:, 1], Bt[:, 2])
    assert slot_dict(*S.residual()) == {(a, b): (c, d) for a, b, c, d in fx["after_apply"]["slots"]}
    _, e = S.vertex_state()
    assert list(e) == fx["after_apply"]["excess"]
    if "heights_after_apply" in fx:
        S.global_relabel()
        h, _ = S.vertex_state()
        assert list(h) == fx["heights_after_apply"]
    S.resolve()
    assert S.query()[0] == fx["value"]
    S.close()


def test_golden_static_init_gpu():
    with open(os.path.join(GOLDEN, "static_init_heights.json")) as fh:
        fx = json.load(fh)
    E = np.array(fx["edges"]).reshape(-1, 3)
    S = native.Solver(fx["n"], E[:, 0], E[:, 1], E[:, 2], fx["s"], fx["t"])
    assert S.query()[0] == fx["value"]
    out = E[:, 0] == fx["s"]
    S.set_flow(E[out, 0], E[out, 1], E[out, 2])
    assert slot_dict(*S.residual()) == {(a, b): (c, d) for a, b, c, d in fx["after_init"]["slots"]}
    S.global_relabel()
    h, e = S.vertex_state()
    assert list(h) == fx["heights"] and list(e) == fx["after_init"]["excess"]
    S.close()


@pytest.mark.parametrize("seed", range(8))
def test_resolve_from_arbitrary_pseudoflow(seed):
    """From any 0 <= f <= c, Alg. 5 (source saturation + loop) reaches the max flow."""
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(3, 1500))
    src, dst, cap = W.random_multigraph(n, 6 * n, seed=900 + seed, cap_hi=40)
    mu, mv, mc = oracle.merge(n, src, dst, cap)
    f = _random_flow(rng, mc, frac=0.9)
    S = native.Solver(n, src, dst, cap, 0, n - 1)
    S.set_flow(mu, mv, f)
    S.update(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32))
    check_against_oracle(S, n, src, dst, cap, 0, n - 1)
    S.close()


# ---------------------------------------------------------------------------
# flow extraction and errors
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("seed", range(6))
def test_get_flow_invariants(seed):
    rng = np.random.default_rng(1000 + seed)
    g = W.erdos_renyi(2500, 15000, seed=1000 + seed, cap_hi=100)
    S, es = run_dynamic(g, lambda es, k: W.mixed_batch(es, 300, rng, ins_cap_hi=100), 2)
    v = S.query()[0]
    before = slot_dict(*S.residual())
    u, vv, cap, f = S.get_flow()
    flow_invariants(g.n, g.s, g.t, u, vv, cap, f, v)
    assert slot_dict(*S.residual()) == before      # extraction works on a copy
    uu, vv2, cc = es.coo()
    keep = cc > 0
    assert sorted(zip(u.tolist(), vv.tolist(), cap.tolist())) == sorted(
        zip(uu[keep].tolist(), vv2[keep].tolist(), cc[keep].tolist()))
    S.close()


def test_invalid_batch_rejected_whole():
    g = W.erdos_renyi(300, 2000, seed=81, cap_hi=50)
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    before = slot_dict(*S.residual())
    for u, v, c in [([1, 2], [3, 300], [5, 5]), ([1, -1], [3, 4], [5, 5]), ([1, 2], [3, 4], [5, -2])]:
        with pytest.raises(native.MaxflowError) as ei:
            S.update(np.array(u), np.array(v), np.array(c))
        assert ei.value.code == native.ERR_INVALID
    assert slot_dict(*S.residual()) == before
    import torch
    with pytest.raises(native.MaxflowError) as ei:   # device batch: rejected by the kernel
        S.update(torch.tensor([1, 2], device="cuda"), torch.tensor([3, 300], device="cuda"),
                 torch.tensor([5, 5], device="cuda"))
    assert ei.value.code == native.ERR_INVALID
    assert slot_dict(*S.residual()) == before
    S.update(np.array([1]), np.array([3]), np.array([7]))      # usable afterwards
    S.close()


def test_pair_sum_limit_refuses_the_whole_batch():
    """Residual capacities are int32 and c_f(u,v) + c_f(v,u) = c(u,v) + c(v,u)
    (Sec. 3.1 Theorem 3.3), so a batch (Sec. 4.1: it sets new capacities) that
    would leave a pair above INT32_MAX is refused before anything changes.  The
    final capacity of both directions counts, the batch's own update of the
    reverse included."""
    M = 2**31 - 1
    # three disjoint paths of capacity INT32_MAX (value 3 * INT32_MAX in int64),
    # and a dead-end pair (1, 4) whose sum is INT32_MAX - 5
    src = [0, 1, 0, 2, 0, 3, 1, 4]
    dst = [1, 5, 2, 5, 3, 5, 4, 1]
    cap = [M, M, M, M, M, M, M - 10, 5]
    n, s, t = 6, 0, 5
    S = native.Solver(n, src, dst, cap, s, t)
    assert S.query()[0] == 3 * M
    before = slot_dict(*S.residual())
    h0, e0 = S.vertex_state()
    over = [
        ([4], [1], [11]),                       # one direction: (M - 10) + 11
        ([1, 4], [4, 1], [M - 7, 8]),           # both: each fits with the other's old value, not together
        ([2, 3], [3, 2], [M, 1]),               # a new pair, both directions in the batch
        ([1, 4, 1], [4, 1, 4], [5, M, M - 10]),  # last update wins: (M - 10) + M
    ]
    for u, v, c in over:
        with pytest.raises(native.MaxflowError) as ei:
            S.update(np.array(u), np.array(v), np.array(c, dtype=np.int64).astype(np.int32))
        assert ei.value.code == native.ERR_TOO_LARGE
        assert slot_dict(*S.residual()) == before
        h1, e1 = S.vertex_state()
        np.testing.assert_array_equal(e1, e0)
        assert S.query()[0] == 3 * M
    import torch
    with pytest.raises(native.MaxflowError) as ei:      # a device batch: refused by the kernel too
        S.update(torch.tensor([4], dtype=torch.int32, device="cuda"), torch.tensor([1], dtype=torch.int32, device="cuda"),
                 torch.tensor([11], dtype=torch.int32, device="cuda"))
    assert ei.value.code == native.ERR_TOO_LARGE
    assert slot_dict(*S.residual()) == before
    # exactly at the limit: accepted, and the value equals Dinic's int64 value
    es = W.EdgeSet(n, np.array(src), np.array(dst), np.array(cap))
    for u, v, c in [([1, 4], [4, 1], [M - 2, 2]), ([2], [3], [M]), ([3, 4], [5, 5], [M, M])]:
        S.update(np.array(u), np.array(v), np.array(c, dtype=np.int64).astype(np.int32))
        es.apply(np.array(u), np.array(v), np.array(c))
        uu, vv, cc = es.coo()
        got = check_against_oracle(S, n, uu, vv, cc, s, t)
        cpu_certificate(S, got)
    assert S.query()[0] == 3 * M               # the source's out-capacity still bounds it
    S.close()


def test_iteration_cap_reports_not_converged():
    g = W.erdos_renyi(3000, 24000, seed=91, cap_hi=100)
    with pytest.raises(native.MaxflowError) as ei:
        native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t, max_iters=1, kernel_cycles=1)
    assert ei.value.code == native.ERR_NOT_CONVERGED


def test_init_rejects_bad_arguments():
    for args in [(3, [0], [1], [1], 0, 0), (3, [0], [5], [1], 0, 2), (3, [0], [1], [-1], 0, 2), (1, [], [], [], 0, 0)]:
        with pytest.raises(native.MaxflowError) as ei:
            native.Solver(*args)
        assert ei.value.code == native.ERR_INVALID


def test_clone_is_independent_deep_copy():
    g = W.erdos_renyi(2000, 14000, seed=131, cap_hi=100)
    rng = np.random.default_rng(132)
    S, es = run_dynamic(g, lambda es, k: W.mixed_batch(es, 300, rng, ins_cap_hi=100), 2)
    C = S.clone()
    assert slot_dict(*C.residual()) == slot_dict(*S.residual())
    assert C.query()[0] == S.query()[0]
    b = W.mixed_batch(es, 400, rng, ins_cap_hi=100, frac=(0.2, 0.2, 0.4))
    es.apply(b.u, b.v, b.cap)
    C.update(b.u, b.v, b.cap)
    u2, v2, c2 = es.coo()
    check_against_oracle(C, g.n, u2, v2, c2, g.s, g.t)
    S.update(b.u, b.v, b.cap)
    assert S.query()[0] == C.query()[0]
    C.close()
    S.close()


@pytest.mark.parametrize("k", [1, 3, 64])
def test_kernel_cycles_do_not_change_the_value(k):
    g = W.erdos_renyi(2500, 16000, seed=141, cap_hi=100)
    rng = np.random.default_rng(142)
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    S.set_kernel_cycles(k)
    assert S.stats()["kernel_cycles"] == k
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    for _ in range(3):
        b = W.mixed_batch(es, 300, rng, ins_cap_hi=100)
        es.apply(b.u, b.v, b.cap)
        S.update(b.u, b.v, b.cap)
        u2, v2, c2 = es.coo()
        check_against_oracle(S, g.n, u2, v2, c2, g.s, g.t)
    S.close()


@pytest.mark.parametrize("rounds,k", [(0, 0), (0, 1), (4, 1), (32, 4), (256, 16)])
def test_discharge_rounds_do_not_change_the_value(rounds, k):
    # rounds 0: the adaptive count (at least 2, more while the discharge is cheap against its BFS)
    g = W.erdos_renyi(3000, 18000, seed=151, cap_hi=100)
    rng = np.random.default_rng(152)
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    S.set_rounds(rounds)
    S.set_kernel_cycles(k)
    S.resolve_static()
    check_against_oracle(S, g.n, g.src, g.dst, g.cap, g.s, g.t)
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    for _ in range(3):
        b = W.mixed_batch(es, 400, rng, ins_cap_hi=100, st_bias=(g.s, g.t, 0.3))
        es.apply(b.u, b.v, b.cap)
        S.update(b.u, b.v, b.cap)
        u2, v2, c2 = es.coo()
        check_against_oracle(S, g.n, u2, v2, c2, g.s, g.t)
    assert S.stats()["rounds"] == rounds
    if rounds == 0:
        assert S.stats()["discharge_rounds"] >= 1
    S.close()


@pytest.mark.parametrize("alpha,beta", [(0, 24), (1, 1), (14, 24), (1000, 1000)])
def test_bfs_direction_switch_does_not_change_labels_or_values(alpha, beta):
    # bottom-up levels label exactly what top-down levels label: same heights after a BFS-only
    # relabel of the same state, and the same values over updates
    g = W.rmat(12, 16, 0.57, 0.19, 0.19, seed=171, cap_hi=1000)
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    rng = np.random.default_rng(172)
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    R = S.clone()
    S.set_bfs_switch(alpha, beta)
    R.set_bfs_switch(0, 24)
    for _ in range(3):
        b = W.mixed_batch(es, 300, rng, ins_cap_hi=1000, st_bias=(g.s, g.t, 0.3))
        es.apply(b.u, b.v, b.cap)
        S.update(b.u, b.v, b.cap)
        R.update(b.u, b.v, b.cap)
        u2, v2, c2 = es.coo()
        check_against_oracle(S, g.n, u2, v2, c2, g.s, g.t)
        assert S.query()[0] == R.query()[0]
    # same state, BFS only: identical heights whatever the direction
    C = S.clone()
    C.set_bfs_switch(0, 24)
    S.global_relabel()
    C.global_relabel()
    assert np.array_equal(S.vertex_state()[0], C.vertex_state()[0])
    with pytest.raises(native.MaxflowError):
        S.set_bfs_switch(-1, 24)
    C.close(); R.close(); S.close()


@pytest.mark.parametrize("family", ["rmat12", "grid64", "geometric"])
def test_one_cta_bfs_levels_give_the_same_heights_and_values(family):
    # small top-down levels run in the first CTA alone (maxflow_set_bfs_tail):
    # the heights of a BFS-only relabel and the values over updates are those of
    # the grid-wide levels, and the oracle's heights
    if family == "rmat12":
        g = W.rmat(12, 16, 0.57, 0.19, 0.19, seed=181, cap_hi=1000)
        mk = lambda es, rng: W.mixed_batch(es, 300, rng, ins_cap_hi=1000, st_bias=(g.s, g.t, 0.3))
    elif family == "grid64":
        G = W.GridSegmentation(side=64, seed=3, window=16, origin=(16, 16), step=1)
        g = G.graph()
        ks = iter(range(30))
        mk = lambda es, rng: G.window_batch(next(ks))
    else:
        g = W.geometric(4000, seed=183)
        mk = lambda es, rng: W.mixed_batch(es, 200, rng, ins_cap_hi=500)
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    rng = np.random.default_rng(182)
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    R = S.clone()
    S.set_bfs_tail(1 << 20)          # every top-down level qualifies
    R.set_bfs_tail(0)
    for _ in range(3):
        b = mk(es, rng)
        es.apply(b.u, b.v, b.cap)
        S.update(b.u, b.v, b.cap)
        R.update(b.u, b.v, b.cap)
        u2, v2, c2 = es.coo()
        check_against_oracle(S, g.n, u2, v2, c2, g.s, g.t)
        assert S.query()[0] == R.query()[0]
    C = S.clone()
    C.set_bfs_tail(0)
    S.global_relabel()
    C.global_relabel()
    h = S.vertex_state()[0]
    assert np.array_equal(h, C.vertex_state()[0])
    su, sv, scap, scf = S.residual()
    Ro = oracle.Residual(g.n, *es.coo())
    _, e = S.vertex_state()
    # the oracle's heights on the same residual state (loaded as a flow)
    flow = np.maximum(scap.astype(np.int64) - scf, 0)
    keep = scap > 0
    Ro.set_flow(su[keep], sv[keep], flow[keep].astype(np.int32))
    assert np.array_equal(h, Ro.heights(g.s, g.t, deficit_roots=True))
    with pytest.raises(native.MaxflowError):
        S.set_bfs_tail(-1)
    C.close(); R.close(); S.close()


@pytest.mark.parametrize("rq,div", [(0, 0), (1, 256), (1, 4)])
def test_requeue_and_cycle_budget_do_not_change_values(rq, div):
    # discharge settings that steer work only: the same values as the oracle
    g = W.rmat(12, 16, 0.57, 0.19, 0.19, seed=191, cap_hi=1000)
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    rng = np.random.default_rng(192)
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    S.set_requeue(rq)
    S.set_cycle_div(div)
    for _ in range(3):
        b = W.mixed_batch(es, 500, rng, ins_cap_hi=1000)
        es.apply(b.u, b.v, b.cap)
        S.update(b.u, b.v, b.cap)
        u2, v2, c2 = es.coo()
        v = check_against_oracle(S, g.n, u2, v2, c2, g.s, g.t)
        cpu_certificate(S, v)
    S.resolve_static()
    check_against_oracle(S, g.n, *es.coo(), g.s, g.t)
    L = native.load()
    assert L.maxflow_set_requeue(S.h, 2) == native.ERR_INVALID
    assert L.maxflow_set_cycle_div(S.h, -1) == native.ERR_INVALID
    S.close()


def test_a_stalled_barrier_times_out_and_leaves_the_context_usable():
    # one CTA never arrives at a grid barrier: the others give up after the
    # context's wait limit, the call reports the failure, and the context still
    # solves correctly afterwards (no hang, no fault)
    import time
    g = W.erdos_renyi(3000, 20000, seed=181, cap_hi=100)
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t, wait_limit_s=0.05)
    L = native.load()
    t0 = time.perf_counter()
    rc = L.maxflow_test_stalled_barrier(S.h, 0)
    assert rc == native.ERR_INTERNAL
    assert time.perf_counter() - t0 < 5.0
    assert L.maxflow_test_stalled_barrier(S.h, 1 << 20) == native.ERR_INVALID
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    rng = np.random.default_rng(182)
    for _ in range(2):
        b = W.mixed_batch(es, 500, rng, ins_cap_hi=100)
        es.apply(b.u, b.v, b.cap)
        S.update(b.u, b.v, b.cap)
        u2, v2, c2 = es.coo()
        check_against_oracle(S, g.n, u2, v2, c2, g.s, g.t)
    S.close()


def test_checkpoint_and_rollback_restore_the_saved_state_exactly():
    # a checkpoint, then an update and a call that fails (a stalled barrier):
    # rollback gives back the checkpointed residuals, heights, excesses and value
    # bit for bit, and the context goes on solving correctly
    g = W.erdos_renyi(3000, 20000, seed=191, cap_hi=100)
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t, wait_limit_s=0.05)
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    rng = np.random.default_rng(192)
    b = W.mixed_batch(es, 400, rng, ins_cap_hi=100)
    es.apply(b.u, b.v, b.cap)
    S.update(b.u, b.v, b.cap)
    with pytest.raises(native.MaxflowError) as ei:
        S.rollback()                                   # nothing to roll back to yet
    assert ei.value.code == native.ERR_STATE
    S.checkpoint()
    saved = (slot_dict(*S.residual()), S.vertex_state(), S.query()[0])
    saved_es = es.copy()
    b2 = W.mixed_batch(es, 600, rng, ins_cap_hi=100, frac=(0.2, 0.2, 0.5))   # insertions too
    es.apply(b2.u, b2.v, b2.cap)
    S.update(b2.u, b2.v, b2.cap)
    L = native.load()
    assert L.maxflow_test_stalled_barrier(S.h, 0) == native.ERR_INTERNAL
    S.rollback()
    assert slot_dict(*S.residual()) == saved[0]
    h, e = S.vertex_state()
    np.testing.assert_array_equal(h, saved[1][0])
    np.testing.assert_array_equal(e, saved[1][1])
    assert S.query()[0] == saved[2]
    with pytest.raises(native.MaxflowError):
        S.rollback()                                   # the checkpoint was used up
    S.update(b2.u, b2.v, b2.cap)                       # the same batch again, from the restored state
    check_against_oracle(S, g.n, *es.coo(), g.s, g.t)
    assert saved_es.m <= es.m
    S.close()
