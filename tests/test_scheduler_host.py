"""The scheduler's offline evaluation, targets and trace collection, on the CPU with stand-ins."""
import numpy as np

from paper_2511_01235_gb300 import scheduler as SCH


class FixedNet:
    """Predicts the given log times whatever the features."""

    def __init__(self, y):
        self.y = np.asarray(y, np.float32)

    def forward(self, X):
        return self.y[: len(X)]


def test_evaluate_sums_the_picked_and_the_fixed_actions():
    A = 20
    rng = np.random.default_rng(3)
    T = rng.uniform(1.0, 9.0, size=(5, A))
    M = np.ones_like(T)
    M[0, 3] = 0                                    # an action not measured for row 0
    y = np.log(T)                                  # a perfect predictor picks the fastest action per row
    r = SCH.evaluate(FixedNet(y), np.zeros((5, 16), np.float32), T, M)
    best = np.where(M > 0, T, np.inf).min(axis=1)
    assert np.isclose(r["learned_ms"], T[np.arange(5), np.argmin(y, axis=1)].sum())
    assert np.isclose(r["paper_ms"], T[:, SCH.ACTION_PAPER].sum())
    assert np.isclose(r["default_ms"], T[:, SCH.ACTION_DEFAULT].sum())
    assert np.isclose(r["best_ms"], best.sum())
    assert sum(r["picks"]) == 5 and len(r["picks"]) == A


def test_targets_are_log_times_clamped_below():
    T = np.array([[1.0, np.e, 0.0, 1e-9]])
    t = SCH.targets(T)
    assert t.dtype == np.float32
    assert np.allclose(t, [[0.0, 1.0, np.log(1e-3), np.log(1e-3)]], atol=1e-6)


class _Clone:
    def __init__(self, parent):
        self.parent = parent
        self.t = None

    def run_action(self, u, v, c, a):
        self.t = self.parent.script(a)

    def stats(self):
        return {"ms_update": self.t}

    def close(self):
        pass


class _Solver:
    """Stands in for native.Solver: each clone's run of action a takes the next
    scripted time of a; the solver records the actions it runs itself."""

    def __init__(self, times):
        self.times = {a: list(ts) for a, ts in times.items()}
        self.ran = []

    def script(self, a):
        return self.times[a].pop(0)

    def features(self, u, v, c):
        return np.zeros(16, np.float32)

    def clone(self):
        return _Clone(self)

    def run_action(self, u, v, c, a):
        self.ran.append(a)


class _Batch:
    u = v = cap = np.zeros(1, np.int32)


def test_collect_keeps_the_fastest_run_and_advances_by_the_best_action():
    """Traces take the fastest of `reps` runs of every action (each on a fresh
    clone), and the stream then advances by the batch's fastest action."""
    acts = [0, 1, 2]
    times = {0: [5.0, 4.0], 1: [2.5, 6.0], 2: [3.0, 2.0]}      # fastest runs: 4.0, 2.5, 2.0
    S = _Solver(times)
    X, T, M = SCH.collect(S, [_Batch()], actions=acts, reps=2)
    assert list(T[0, :3]) == [4.0, 2.5, 2.0] and list(M[0, :3]) == [1.0, 1.0, 1.0]
    assert M[0, 3:].sum() == 0                                  # actions not run stay masked
    assert S.ran == [2]
    assert all(len(v) == 0 for v in S.times.values())           # two runs of every action
