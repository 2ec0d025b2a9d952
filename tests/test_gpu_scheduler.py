"""The scheduler network's kernels against the numpy restatement, and the
learned schedule against the fixed ones.

Forward, gradient and one Adam step of the CUDA network agree with the
float64 restatement in oracle/mlp_ref.py to fp32 rounding.  Running updates
through maxflow_update_scheduled never changes the flow value, and with the
committed weights the learned schedule spends less device time than the
paper's fixed schedule (one discharge round, KERNEL_CYCLES = average degree,
Alg. 3) and no more than the library's default schedule on held-out batches it
was not trained on (device time per update call, from CUDA events).
"""
import os

import numpy as np
import pytest

import oracle
from oracle import mlp_ref as R
from paper_2511_01235_gb300 import native
from paper_2511_01235_gb300 import scheduler as SCH
from paper_2511_01235_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _data(seed, n_in, n_out, rows):
    rng = np.random.default_rng(seed)
    x = rng.normal(0, 1, (rows, n_in)).astype(np.float32)
    t = rng.normal(0, 1, (rows, n_out)).astype(np.float32)
    m = (rng.random((rows, n_out)) < 0.8).astype(np.float32)
    m[0, 0] = 1
    return x, t, m


@pytest.mark.parametrize("shape", [(16, 64, 20), (5, 33, 7)])
def test_forward_and_gradient_match_numpy(shape):
    n_in, H, n_out = shape
    mlp = native.MLP(n_in, H, n_out, seed=7)
    p = mlp.params.astype(np.float64)
    x, t, m = _data(1, n_in, n_out, 37)
    y = mlp.forward(x)
    y_ref, _ = R.forward(p, x, n_in, H, n_out)
    np.testing.assert_allclose(y, y_ref, rtol=1e-4, atol=1e-4)
    g, loss = mlp.grad(x, t, m)
    g_ref = R.grad(p, x, t, m, n_in, H, n_out)
    assert loss == pytest.approx(R.loss(p, x, t, m, n_in, H, n_out), rel=1e-4)
    np.testing.assert_allclose(g, g_ref, rtol=2e-3, atol=2e-5 * np.abs(g_ref).max())
    mlp.close()


def test_one_adam_step_matches_numpy():
    n_in, H, n_out = 16, 64, 20
    mlp = native.MLP(n_in, H, n_out, seed=9)
    p0 = mlp.params.astype(np.float64)
    x, t, m = _data(2, n_in, n_out, 50)
    mlp.train(x, t, m, steps=1, lr=1e-2)
    p_ref, _, _ = R.adam_step(p0, R.grad(p0, x, t, m, n_in, H, n_out), np.zeros_like(p0), np.zeros_like(p0), 1, 1e-2)
    np.testing.assert_allclose(mlp.params, p_ref, rtol=1e-4, atol=2e-5)
    mlp.close()


def test_training_lowers_the_loss():
    n_in, H, n_out = 16, 64, 20
    mlp = native.MLP(n_in, H, n_out, seed=3)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(200, n_in)).astype(np.float32)
    w = rng.normal(size=(n_in, n_out)).astype(np.float32)
    t = np.tanh(x @ w).astype(np.float32)
    m = np.ones_like(t)
    _, l0 = mlp.grad(x, t, m)
    l1 = mlp.train(x, t, m, steps=400, lr=3e-3)
    assert l1 < 0.2 * l0
    mlp.close()


def test_scheduled_updates_keep_the_flow_exact():
    g = W.erdos_renyi(2000, 14000, seed=171, cap_hi=100)
    mlp = native.MLP(16, 64, len(native.maxflow_sched_actions()), seed=5)   # untrained: any action must be exact
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    rng = np.random.default_rng(172)
    seen = set()
    for _ in range(5):
        b = W.mixed_batch(es, int(rng.integers(10, 1500)), rng, ins_cap_hi=100)
        es.apply(b.u, b.v, b.cap)
        seen.add(S.update_scheduled(b.u, b.v, b.cap, mlp))
        u2, v2, c2 = es.coo()
        assert S.query()[0] == oracle.maxflow(g.n, u2, v2, c2, g.s, g.t).value
    for a in range(len(native.maxflow_sched_actions())):   # and every action of the table
        C = S.clone()
        b = W.mixed_batch(es.copy(), 300, np.random.default_rng(a), ins_cap_hi=100)
        C.run_action(b.u, b.v, b.cap, a)
        es2 = es.copy()
        es2.apply(b.u, b.v, b.cap)
        u2, v2, c2 = es2.coo()
        assert C.query()[0] == oracle.maxflow(g.n, u2, v2, c2, g.s, g.t).value, a
        C.close()
    S.close()
    mlp.close()


@pytest.mark.skipif(not os.path.exists(SCH.DEFAULT_WEIGHTS), reason="no trained scheduler weights")
def test_learned_schedule_beats_the_fixed_schedules_on_heldout_batches():
    """Held-out streams (seeds the network was not trained on) of mixed batch
    sizes.  Every batch meets the three schedules in the same state: each one
    runs on its own clone of the stream's solver (a clone carries the features
    of the last solves too), twice, and the faster of the two device times
    counts (CUDA events around the call on the clone's stream, the learned
    path's features and forward pass included); the stream's solver then takes
    the batch with the default schedule.  The learned schedule's total is below
    the paper's fixed schedule by a wide margin and no more than 2 % above the
    library's own default schedule.  That bound is loose on purpose: the
    committed weights measure 0.86-0.90 of the default here, but weights trained
    on single-run timings measured 0.92-0.98, and a bound tighter than the
    run-to-run spread would test the noise.  The flow value is the same
    whatever the schedule."""
    import torch
    mlp = SCH.load()
    totals = {"learned": 0.0, "paper": 0.0, "default": 0.0}
    for name, seed, k in [("er4096", 301, 8), ("grid256", 305, 4), ("rmat16", 303, 8), ("rmat18", 304, 8)]:
        g, make = SCH.family(name, seed)
        batches = make(k)
        S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
        for b in batches:
            values = set()
            for key in totals:
                best = float("inf")
                for _ in range(2):
                    C = S.clone()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(C.stream)
                    if key == "learned":
                        C.update_scheduled(b.u, b.v, b.cap, mlp)
                    else:
                        C.run_action(b.u, b.v, b.cap, SCH.ACTION_PAPER if key == "paper" else SCH.ACTION_DEFAULT)
                    e1.record(C.stream)
                    e1.synchronize()
                    best = min(best, e0.elapsed_time(e1))
                    values.add(C.query()[0])
                    C.close()
                totals[key] += best
            assert len(values) == 1                 # same flow value whatever the schedule
            S.run_action(b.u, b.v, b.cap, SCH.ACTION_DEFAULT)
        S.close()
    print("scheduler totals (device ms):", totals)
    assert totals["learned"] < 0.8 * totals["paper"], totals
    assert totals["learned"] < 1.02 * totals["default"], totals
