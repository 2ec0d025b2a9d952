"""The scheduler's offline evaluation and targets, on the CPU with a stand-in network."""
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
