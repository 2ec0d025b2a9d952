"""The residual Bi-CSR (Sec. 5.1) the library builds, checked on the CPU.

maxflow_build_layout runs the same host builder maxflow_init uses, without a
GPU.  Its used slots must equal the oracle's residual state slot for slot:
self-loops dropped, parallel edges summed, one slot at each end of every pair
with an edge in either direction, rows sorted by head.  The reverse index and
the pair capacities must be consistent, and each row's slack must follow
max(slack_min, ceil(deg * slack_factor)).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2511_01235_gb300 import native
from paper_2511_01235_gb300 import workloads as W


def _check_layout(n, src, dst, cap, factor, smin):
    L = native.build_layout(n, src, dst, cap, slack_factor=factor, slack_min=smin)
    off, deg = L["off"], L["deg"]
    R = oracle.Residual(n, src, dst, cap)
    ou, ov, ocap, _ = R.slots()
    got_u, got_v, got_c = [], [], []
    for u in range(n):
        lo, d = int(off[u]), int(deg[u])
        row = slice(lo, lo + d)
        heads = L["dst"][row]
        assert np.all(np.diff(heads) > 0)                     # sorted, one slot per head
        got_u += [u] * d
        got_v += list(heads)
        got_c += list(L["cap"][row])
        # slack: max(slack_min, ceil(deg * factor)), the row rounded up to a multiple of
        # 4 slots (rows start on 16-byte boundaries); slack slots point at themselves
        want_slack = max(smin, math.ceil(d * np.float32(factor)))
        assert lo % 4 == 0
        assert int(off[u + 1]) - lo == -(-(d + want_slack) // 4) * 4
        for x in range(lo + d, int(off[u + 1])):
            assert (L["dst"][x], L["cap"][x], L["rev"][x], L["pcap"][x]) == (u, 0, x, 0)
        for j in range(d):
            x = lo + j
            y = int(L["rev"][x])
            v = int(heads[j])
            assert off[v] <= y < off[v] + deg[v] and L["dst"][y] == u and L["rev"][y] == x
            assert L["pcap"][x] == L["cap"][x] + L["cap"][y]
    assert got_u == list(map(int, ou)) and got_v == list(map(int, ov)) and got_c == list(map(int, ocap))
    return L


@pytest.mark.parametrize("seed", range(25))
def test_layout_equals_the_oracles_slots(seed):
    rng = np.random.default_rng(3000 + seed)
    n = int(rng.integers(2, 60))
    m = int(rng.integers(0, 5 * n))
    src, dst, cap = W.random_multigraph(n, m, seed=3000 + seed, cap_hi=20)   # loops, parallel, zero caps
    factor = float(rng.choice([0.0, 0.25, 0.5, 1.0]))
    smin = int(rng.integers(0, 5))
    _check_layout(n, src, dst, cap, factor, smin)


def test_layout_of_generated_workloads():
    for g in (W.erdos_renyi(500, 3000, seed=5, cap_hi=100), W.rmat(10, 8, 0.57, 0.19, 0.19, seed=6, cap_hi=50),
              W.layered_dag(300, seed=7)):
        L = _check_layout(g.n, g.src, g.dst, g.cap, 0.25, 4)
        assert int(L["deg"].sum()) == oracle.Residual(g.n, g.src, g.dst, g.cap).slots()[0].size


def test_layout_errors():
    lib = native.load()
    S = np.zeros(1, np.int64)
    src, dst, cap = np.array([0, 1], np.int32), np.array([1, 2], np.int32), np.array([3, 4], np.int32)
    p = native._p
    call = lambda n, c, *out: lib.maxflow_build_layout(n, 2, p(src), p(dst), p(c), 0.25, 4, p(S), *out)
    assert call(1, cap, None, None, None, None, None, None) == native.ERR_INVALID           # n < 2
    assert call(2, cap, None, None, None, None, None, None) == native.ERR_INVALID           # vertex 2 out of range
    bad = np.array([3, -1], np.int32)
    assert call(3, bad, None, None, None, None, None, None) == native.ERR_INVALID           # negative capacity
    assert call(3, cap, None, None, None, None, None, None) == native.OK
    need = int(S[0])
    assert need == 8 + 8 + 8                    # slots (0,1) (1,0) (1,2) (2,1), slack 4 per row, rows of 4k
    small = np.zeros(need - 1, np.int32)
    S[0] = need - 1
    assert call(3, cap, None, None, p(small), None, None, None) == native.ERR_INVALID     # array too short
    assert int(S[0]) == need and not small.any()
    assert lib.maxflow_build_layout(3, 2, p(src), p(dst), p(cap), -1.0, 4, p(S), None, None, None, None, None,
                                    None) == native.ERR_INVALID
    assert lib.maxflow_build_layout(3, 2, p(src), p(dst), p(cap), 0.25, 4, None, None, None, None, None, None,
                                    None) == native.ERR_INVALID


def test_a_pair_whose_capacities_overflow_int32_is_too_large():
    big = np.iinfo(np.int32).max
    src, dst = np.array([0, 1, 1], np.int32), np.array([1, 0, 2], np.int32)
    ok = native.build_layout(3, src, dst, np.array([big - 5, 5, 1], np.int32))     # sum = INT32_MAX exactly
    x = int(ok["off"][0])
    assert ok["pcap"][x] == big
    with pytest.raises(native.MaxflowError) as ei:
        native.build_layout(3, src, dst, np.array([big - 5, 6, 1], np.int32))    # one more overflows
    assert ei.value.code == native.ERR_TOO_LARGE
    # parallel edges are summed before the pair is checked
    with pytest.raises(native.MaxflowError) as ei:
        native.build_layout(2, np.array([0, 0], np.int32), np.array([1, 1], np.int32),
                            np.array([big, 1], np.int32))
    assert ei.value.code == native.ERR_TOO_LARGE


def test_layout_at_scale_equals_the_oracle_vectorised():
    # R-MAT scale 16 (65,536 vertices, ~1 M edges): the multi-threaded row pass of
    # the builder against the oracle's slots, checked with whole-array operations
    g = W.rmat(16, 16, 0.57, 0.19, 0.19, seed=41, cap_hi=1000)
    L = native.build_layout(g.n, g.src, g.dst, g.cap)
    off, deg = L["off"].astype(np.int64), L["deg"].astype(np.int64)
    used = np.concatenate([np.arange(o, o + d) for o, d in zip(off[:-1], deg)]) if g.n else np.zeros(0, np.int64)
    row = np.repeat(np.arange(g.n), deg)
    ou, ov, ocap, _ = oracle.Residual(g.n, g.src, g.dst, g.cap).slots()
    assert np.array_equal(row, ou) and np.array_equal(L["dst"][used], ov) and np.array_equal(L["cap"][used], ocap)
    rev = L["rev"][used].astype(np.int64)
    assert np.array_equal(L["rev"][rev], used)                     # an involution on the used slots
    assert np.array_equal(L["dst"][rev], row)                      # the reverse slot points back
    assert np.array_equal(L["pcap"][used], L["cap"][used] + L["cap"][rev])
    want = deg + np.maximum(4, np.ceil(deg * 0.25).astype(np.int64))
    assert np.array_equal(off[1:] - off[:-1], (want + 3) // 4 * 4)       # rows of a multiple of 4 slots
    assert np.all(off % 4 == 0)
