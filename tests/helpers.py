"""Shared test helpers: CPU-side checks of a downloaded GPU state.

These checks are written from the definitions (Sec. 2.1 flow constraints,
Sec. 3.1 Theorem 3.3 pair sums, Theorem 3.4 cut certificate) with numpy; they
share no code with the CUDA library or the oracle.
"""
import numpy as np


def slot_dict(u, v, cap, cf):
    return {(int(a), int(b)): (int(c), int(d)) for a, b, c, d in zip(u, v, cap, cf)}


def certificate(n, s, t, su, sv, scap, scf, h, e, value):
    """Check that (residual, heights, excess) certify `value` as the max flow.

    - every slot has its reverse, c_f >= 0 and c_f(u,v) + c_f(v,u) = c(u,v) + c(v,u)
    - e(x) = sum over x's slots of c_f - c (net inflow)
    - A = {h == n} holds s, not t; no residual slot leads from A out of A
    - no active vertex: e(x) <= 0 for x not in A, x != t
    - C(A, V \\ A) = value = sum of e over V \\ A
    Returns a dict of counts (all zero on success) plus the cut capacity.
    """
    su = np.asarray(su, np.int64)
    sv = np.asarray(sv, np.int64)
    scap = np.asarray(scap, np.int64)
    scf = np.asarray(scf, np.int64)
    h = np.asarray(h, np.int64)
    e = np.asarray(e, np.int64)
    key = su * n + sv
    rkey = sv * n + su
    order = np.argsort(key)
    ks = key[order]
    pos = np.searchsorted(ks, rkey)
    pos = np.minimum(pos, ks.size - 1)
    has_rev = ks[pos] == rkey
    ridx = order[pos]
    pair_bad = int((~has_rev).sum())
    ok = has_rev
    pair_bad += int(((scf[ok] + scf[ridx[ok]]) != (scap[ok] + scap[ridx[ok]])).sum())
    neg = int((scf < 0).sum())
    ex = np.bincount(su, weights=(scf - scap).astype(np.float64), minlength=n)
    # float64 sums are exact here (|values| < 2^53)
    ex_bad = int((ex.astype(np.int64) != e).sum())
    A = h == n
    cross = A[su] & ~A[sv]
    cross_res = int((cross & (scf > 0)).sum())
    cut = int(scap[cross].sum())
    act = ~A & (e > 0)
    act[t] = False
    val_b = int(e[~A].sum())
    return {
        "pair_bad": pair_bad,
        "neg": neg,
        "excess_bad": ex_bad,
        "s_not_in_A": int(not A[s]),
        "t_in_A": int(A[t]),
        "cross_residual": cross_res,
        "active": int(act.sum()),
        "cut_ne_value": int(cut != value),
        "valueB_ne_value": int(val_b != value),
        "cut": cut,
    }


def assert_certificate(n, s, t, su, sv, scap, scf, h, e, value):
    r = certificate(n, s, t, su, sv, scap, scf, h, e, value)
    bad = {k: v for k, v in r.items() if k != "cut" and v}
    assert not bad, (bad, r["cut"], value)
    return r


def flow_invariants(n, s, t, u, v, cap, f, value):
    """0 <= f <= cap on every edge, conservation off {s,t}, net out of s = net into t = value."""
    u = np.asarray(u, np.int64)
    v = np.asarray(v, np.int64)
    cap = np.asarray(cap, np.int64)
    f = np.asarray(f, np.int64)
    assert np.all(f >= 0) and np.all(f <= cap)
    inflow = np.bincount(v, weights=f.astype(np.float64), minlength=n).astype(np.int64)
    outflow = np.bincount(u, weights=f.astype(np.float64), minlength=n).astype(np.int64)
    net = inflow - outflow
    mask = np.ones(n, bool)
    mask[[s, t]] = False
    bad = np.flatnonzero(net[mask] != 0)
    assert bad.size == 0, ("conservation", bad[:10])
    assert -net[s] == value, (-net[s], value)
    assert net[t] == value, (net[t], value)
