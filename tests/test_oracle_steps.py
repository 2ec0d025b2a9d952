"""Single steps of the oracle against hand-derived fixtures (tests/golden/steps_*).

Between two global relabels, the sequential restatement only raises heights
and pushes downhill, so it never makes a steep residual edge: Alg. 3 (and its
pull mirror) never fires inside the loop, and relabel details do not change
the final value.  These fixtures run Alg. 2 on one vertex, Alg. 3, and their
pull mirrors (Sec. 5.2.2, reading R8) from heights the test sets.  After each
step they check every c_f, excess and height, and the push and relabel
counts, against values derived by hand in the fixture.
"""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _state(R):
    u, v, cap, cf = R.slots()
    e, h = R.vertex()
    return [(int(a), int(b), int(c)) for a, b, c in zip(u, v, cap)], [int(x) for x in cf], list(map(int, e)), \
        list(map(int, h))


def _check_invariants(fx, slots, cf, e):
    # pair sums c_f(u,v) + c_f(v,u) = c(u,v) + c(v,u), excess from its definition, excess sums to 0
    idx = {(u, v): k for k, (u, v, _) in enumerate(slots)}
    for k, (u, v, c) in enumerate(slots):
        r = idx[(v, u)]
        assert cf[k] + cf[r] == c + slots[r][2]
    for x in range(fx["n"]):
        assert e[x] == sum(cf[k] - slots[k][2] for k, (u, _, _) in enumerate(slots) if u == x)
    assert sum(e) == 0


@pytest.mark.parametrize("name", ["steps_push_discharge_remove_invalid.json",
                                  "steps_pull_discharge_remove_invalid.json"])
def test_single_steps_match_the_hand_derivation(name):
    fx = _load(name)
    E = np.array(fx["edges"]).reshape(-1, 3)
    R = oracle.Residual(fx["n"], E[:, 0], E[:, 1], E[:, 2])
    s, t = fx["s"], fx["t"]
    if fx["start"] == "static_init":
        R.static_init(s)
    slots, cf, e, _ = _state(R)
    assert slots == [tuple(x) for x in fx["slots"]]
    assert cf == fx["start_state"]["cf"] and e == fx["start_state"]["excess"]
    for k, op in enumerate(fx["ops"]):
        kind = op["op"]
        if kind == "set_heights":
            R.set_heights(op["h"])
            continue
        if kind == "discharge":
            pushes, relabels = R.discharge(op["u"], op["cycles"])
            assert (pushes, relabels) == (op["pushes"], op["relabels"]), (k, kind)
        elif kind == "remove_invalid":
            R.remove_invalid(s, t)
        elif kind == "pull_discharge":
            R.pull_discharge(op["u"], op["cycles"])
        elif kind == "pull_remove_invalid":
            R.pull_remove_invalid(s, t)
        elif kind == "saturate_sink":
            R.saturate_sink(t)
        elif kind == "pull_heights":
            assert list(map(int, R.pull_heights(s, t))) == op["heights"], (k, kind)
        else:
            raise AssertionError(kind)
        _, cf, e, h = _state(R)
        if "cf" in op:
            assert cf == op["cf"], (k, kind)
        if "excess" in op:
            assert e == op["excess"], (k, kind)
        if "heights" in op:
            assert h == op["heights"], (k, kind)
        _check_invariants(fx, slots, cf, e)


def test_set_heights_rejects_out_of_range():
    R = oracle.Residual(3, [0, 1], [1, 2], [1, 1])
    with pytest.raises(ValueError):
        R.set_heights([0, 4, 0])
    with pytest.raises(ValueError):
        R.set_heights([0, 1])


def test_sequential_loop_is_the_single_steps_composed():
    # one outer iteration of the sequential loop = BFS heights, Alg. 2 on each
    # active vertex in increasing id order, then Alg. 3 (Alg. 1 / Alg. 5 loop)
    rng = np.random.default_rng(77)
    for trial in range(20):
        n = int(rng.integers(4, 40))
        m = int(rng.integers(n, 4 * n))
        src = rng.integers(0, n, m)
        dst = rng.integers(0, n, m)
        cap = rng.integers(0, 20, m)
        s, t = 0, n - 1
        A = oracle.Residual(n, src, dst, cap)
        B = oracle.Residual(n, src, dst, cap)
        A.static_init(s)
        B.static_init(s)
        kc = int(rng.integers(1, 5))
        try:
            A.push_relabel(s, t, kernel_cycles=kc, max_iters=1)
        except RuntimeError:
            pass                                    # one iteration rarely converges
        h = B.heights(s, t)
        e, _ = B.vertex()
        active = [x for x in range(n) if x not in (s, t) and e[x] > 0 and h[x] < n]
        if active:
            for u in active:
                B.discharge(u, kc)
            B.remove_invalid(s, t)
        _, cfa, ea, ha = _state(A)
        _, cfb, eb, hb = _state(B)
        assert (cfa, ea, ha) == (cfb, eb, hb), trial
