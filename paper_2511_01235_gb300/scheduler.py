"""Learned schedule for incremental max-flow updates.

The solver's work per update depends on a few knobs the paper fixes by hand:
KERNEL_CYCLES (Sec. 6.1: the average degree), how often the global relabel
runs, and whether to repair the flow incrementally at all (Sec. 6.2: past a
graph-dependent batch size the static solve wins).  A schedule (action) sets
all three; the table is fixed in the library (maxflow_sched_actions).  A small
network (maxflow_mlp_*: 16 -> 64 -> 64 -> one output per action) predicts the
log device time of every action from the batch's features; the scheduler
runs the action with the smallest prediction.  The flow value never depends
on the schedule.

Training data are the solver's own traces: for each (state, batch) the batch is
run once per action on a clone of the state, and the device time recorded.
Training runs on the GPU through the library's forward/backward/Adam kernels.

    python -m paper_2511_01235_gb300.scheduler --out paper_2511_01235_gb300/scheduler_weights.json
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import native
from . import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "scheduler_weights.json")
ACTION_DEFAULT = 0     # the library's default schedule (adaptive rounds, KERNEL_CYCLES = average degree)
ACTION_PAPER = 5       # one discharge round, KERNEL_CYCLES = average degree, Alg. 3 (the paper's schedule)
N_FEATURES = 16


# ---------------------------------------------------------------------------
# workloads the traces come from
# ---------------------------------------------------------------------------

def _sizes(rng, lo, hi, k):
    return [int(x) for x in np.exp(rng.uniform(math.log(lo), math.log(hi), size=k))]


def family(name: str, seed: int):
    """(graph, batch maker) for one workload family; the maker yields update batches."""
    rng = np.random.default_rng(seed)
    if name.startswith("er"):
        n = int(name[2:] or 4096)
        g = W.erdos_renyi(n, 8 * n, seed=seed, cap_hi=100)
        es = W.EdgeSet(g.n, g.src, g.dst, g.cap)

        def make(k):
            out = []
            for B in _sizes(rng, 16, es.m // 8, k):
                kind = rng.integers(0, 4)
                if kind == 0:
                    b = W.mixed_batch(es, B, rng, ins_cap_hi=100)
                elif kind == 1:
                    b = W.kind_batch(es, B, rng, "inc")
                elif kind == 2:
                    b = W.kind_batch(es, B, rng, "dec")
                else:
                    b = W.mixed_batch(es, B, rng, ins_cap_hi=100, st_bias=(g.s, g.t, 0.3))
                es.apply(b.u, b.v, b.cap)
                out.append(b)
            return out
        return g, make
    if name.startswith("rmat"):
        scale = int(name[4:] or 18)
        g = W.rmat(scale, 16, 0.57, 0.19, 0.19, seed=seed, cap_hi=1000)
        es = W.EdgeSet(g.n, g.src, g.dst, g.cap)

        def make(k):
            out = []
            for B in _sizes(rng, 100, min(200_000, es.m // 8), k):
                b = W.mixed_batch(es, B, rng, ins_cap_hi=1000,
                                  st_bias=(g.s, g.t, 0.3) if rng.random() < 0.3 else None)
                es.apply(b.u, b.v, b.cap)
                out.append(b)
            return out
        return g, make
    if name.startswith("grid"):
        side = int(name[4:] or 256)
        w = min(256, side // 4)
        G = W.GridSegmentation(side=side, seed=seed, window=w, origin=(side // 4, side // 4),
                               step=max(1, w // 32))
        g = G.graph()
        state = {"k": int(rng.integers(0, 8))}

        def make(k):
            out = []
            for _ in range(k):
                out.append(G.window_batch(state["k"] % 30))
                state["k"] += 1
            return out
        return g, make
    raise ValueError(name)


# ---------------------------------------------------------------------------
# traces
# ---------------------------------------------------------------------------

def collect(solver: native.Solver, batches, actions=None, log=None, reps=1):
    """Features and per-action device time (ms) of every batch, each action on a
    clone (the fastest of `reps` runs, each on a fresh clone: single runs vary
    by several percent, and a noisy target teaches the network noise).  The
    state then advances by the batch's fastest action: the states a good
    schedule meets are those it makes itself, and a static re-solve or a
    many-round update leaves a different preflow than the default would."""
    if actions is None:
        actions = list(range(len(native.maxflow_sched_actions())))
    A = len(native.maxflow_sched_actions())
    X = np.zeros((len(batches), N_FEATURES), np.float32)
    T = np.zeros((len(batches), A), np.float64)
    M = np.zeros((len(batches), A), np.float32)
    for i, b in enumerate(batches):
        X[i] = solver.features(b.u, b.v, b.cap)
        for a in actions:
            t = float("inf")
            for _ in range(max(1, reps)):
                C = solver.clone()
                C.run_action(b.u, b.v, b.cap, a)
                t = min(t, C.stats()["ms_update"])
                C.close()
            T[i, a] = t
            M[i, a] = 1.0
        solver.run_action(b.u, b.v, b.cap, int(np.argmin(np.where(M[i] > 0, T[i], np.inf))))
        if log:
            log(f"  batch {i} B={b.size} best action {int(np.argmin(np.where(M[i] > 0, T[i], np.inf)))} "
                f"{T[i][M[i] > 0].min():.3f} ms, paper {T[i, ACTION_PAPER]:.3f} ms")
    return X, T, M


def collect_family(name, seed, k, log=None, reps=1):
    g, make = family(name, seed)
    S = native.Solver(g.n, g.src, g.dst, g.cap, g.s, g.t)
    batches = make(k)
    X, T, M = collect(S, batches, log=log, reps=reps)
    S.close()
    return X, T, M


# ---------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------

def targets(T):
    return np.log(np.maximum(T, 1e-3)).astype(np.float32)


def train(X, T, M, hidden=64, steps=3000, lr=3e-3, seed=0):
    mlp = native.MLP(N_FEATURES, hidden, T.shape[1], seed=seed)
    loss = mlp.train(X, targets(T), M, steps=steps, lr=lr)
    return mlp, loss


def save(mlp: native.MLP, path, meta=None):
    doc = {"n_in": mlp.n_in, "n_hidden": mlp.n_hidden, "n_out": mlp.n_out,
           "actions": native.maxflow_sched_actions(), "params": [float(x) for x in mlp.params]}
    if meta:
        doc["meta"] = meta
    with open(path, "w") as f:
        json.dump(doc, f)


def load(path=DEFAULT_WEIGHTS) -> native.MLP:
    with open(path) as f:
        doc = json.load(f)
    acts = [tuple(a) for a in doc["actions"]]
    if acts != [tuple(a) for a in native.maxflow_sched_actions()]:
        raise ValueError("scheduler weights were trained for a different action table")
    mlp = native.MLP(doc["n_in"], doc["n_hidden"], doc["n_out"])
    mlp.params = np.asarray(doc["params"], np.float32)
    return mlp


def evaluate(mlp: native.MLP, X, T, M):
    """Offline: total time of the predicted actions vs the fixed schedules vs the best action."""
    y = mlp.forward(X)
    pick = np.argmin(y, axis=1)
    rows = np.arange(len(X))
    return {"learned_ms": float(T[rows, pick].sum()), "paper_ms": float(T[:, ACTION_PAPER].sum()),
            "default_ms": float(T[:, ACTION_DEFAULT].sum()),
            "best_ms": float(np.where(M > 0, T, np.inf).min(axis=1).sum()),
            "picks": np.bincount(pick, minlength=T.shape[1]).tolist()}


TRAIN_PLAN = [("er4096", 101, 24), ("er16384", 102, 16), ("rmat16", 103, 20), ("rmat18", 104, 20),
              ("rmat20", 2, 16), ("grid256", 105, 10), ("grid512", 106, 6)]
HELDOUT_PLAN = [("er4096", 201, 12), ("rmat16", 203, 8), ("rmat18", 204, 8), ("grid256", 205, 6)]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--traces", default=None, help="save traces (npz) here")
    ap.add_argument("--reps", type=int, default=2, help="runs per action and batch (the fastest counts)")
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    native.load()
    t0 = time.time()
    parts = []
    for name, seed, k in TRAIN_PLAN:
        print(f"collect {name} seed {seed} x{k}", flush=True)
        parts.append(collect_family(name, seed, k, log=print, reps=args.reps))
    X = np.concatenate([p[0] for p in parts])
    T = np.concatenate([p[1] for p in parts])
    M = np.concatenate([p[2] for p in parts])
    held = [collect_family(name, seed, k, reps=args.reps) for name, seed, k in HELDOUT_PLAN]
    Xh = np.concatenate([p[0] for p in held])
    Th = np.concatenate([p[1] for p in held])
    Mh = np.concatenate([p[2] for p in held])
    if args.traces:
        np.savez(args.traces, X=X, T=T, M=M, Xh=Xh, Th=Th, Mh=Mh)
    mlp, loss = train(X, T, M, steps=args.steps)
    ev_train = evaluate(mlp, X, T, M)
    ev_held = evaluate(mlp, Xh, Th, Mh)
    meta = {"train_rows": int(len(X)), "train_loss": loss, "train_eval": ev_train, "heldout_eval": ev_held,
            "collect_s": time.time() - t0, "plan": TRAIN_PLAN, "reps": args.reps}
    save(mlp, args.out, meta)
    print(json.dumps(meta), flush=True)


if __name__ == "__main__":
    main()
