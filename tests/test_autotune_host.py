"""The autotuner's coordinate descent, on the CPU with a synthetic cost.

The batched launch is replaced by a function of the knobs the tuner set on
the solvers, so the search itself is checked: it finds the best value of
every knob when the cost is separable, never returns a configuration worse
than the default, stops after a pass without gain, does not keep a
configuration that won one trial by luck, and leaves the solvers set to what
it returns.
"""
from paper_2511_01235_gb300 import autotune, native


class FakeSolver:
    def __init__(self):
        self.rounds = self.cycles = None
        self.split = None

    def set_rounds(self, r):
        self.rounds = r

    def set_kernel_cycles(self, k):
        self.cycles = k

    def set_tuning(self, *split):
        self.split = tuple(split)


def _install(monkeypatch, cost):
    calls = []

    def fake_batched(solvers, batches, group_blocks=8):
        s = solvers[0]
        assert all((x.rounds, x.cycles, x.split) == (s.rounds, s.cycles, s.split) for x in solvers)
        calls.append((group_blocks, s.rounds, s.cycles, s.split))
        return cost(group_blocks, s.rounds, s.cycles, s.split)

    monkeypatch.setattr(native, "maxflow_solve_batched", fake_batched)
    return calls


def test_separable_cost_reaches_the_optimum(monkeypatch):
    want = {"group_blocks": 4, "rounds": 16, "cycles": 4, "split": autotune.SPLITS[2]}

    def cost(gb, r, k, sp):
        return (10.0 + abs(autotune.GROUP_BLOCKS.index(gb) - 2) + abs(autotune.ROUNDS.index(r) - 3)
                + abs(autotune.CYCLES.index(k) - 1) + abs(autotune.SPLITS.index(sp) - 2))

    _install(monkeypatch, cost)
    S = [FakeSolver() for _ in range(3)]
    best, best_ms, trials = autotune.tune(S, passes=3, reps=1)
    assert best == want and best_ms == 10.0
    assert all((s.rounds, s.cycles, s.split) == (16, 4, autotune.SPLITS[2]) for s in S)
    assert min(ms for _, ms in trials) == best_ms


def test_never_worse_than_the_default_and_stops_without_gain(monkeypatch):
    calls = _install(monkeypatch, lambda gb, r, k, sp: 5.0 if (gb, r, k, sp) == (8, 0, 0, (0, 0, 0)) else 7.0)
    S = [FakeSolver()]
    best, best_ms, trials = autotune.tune(S, passes=4, reps=2)
    assert best == autotune.DEFAULT and best_ms == 5.0
    # one pass over every other value of every knob, then stop (no gain)
    others = sum(len(v) - 1 for v in (autotune.GROUP_BLOCKS, autotune.ROUNDS, autotune.CYCLES, autotune.SPLITS))
    assert len(trials) == 1 + others
    assert len(calls) == 2 * (1 + others)                 # reps launches per trial


def test_a_lucky_trial_does_not_replace_the_default(monkeypatch):
    """A configuration that wins its one descent trial but loses the interleaved
    confirmation against the default is dropped: the default stays."""
    lucky = (8, 4, 0, (0, 0, 0))          # rounds = 4
    seen = {"lucky": 0}

    def cost(gb, r, k, sp):
        if (gb, r, k, sp) == lucky:
            seen["lucky"] += 1
            return 4.0 if seen["lucky"] <= 2 else 6.0     # fast in its trial (two reps), slow afterwards
        return 5.0 if (gb, r, k, sp) == (8, 0, 0, (0, 0, 0)) else 7.0

    _install(monkeypatch, cost)
    S = [FakeSolver()]
    best, best_ms, trials = autotune.tune(S, passes=2, reps=2, confirm_reps=3)
    assert any(cfg["rounds"] == 4 and ms == 4.0 for cfg, ms in trials)    # it did win its trial
    assert best == autotune.DEFAULT and best_ms == 5.0
    assert (S[0].rounds, S[0].cycles, S[0].split) == (0, 0, (0, 0, 0))


def test_a_win_within_the_margin_is_not_taken(monkeypatch):
    """A trial 1 % faster than the best so far (inside MARGIN) does not replace it."""
    _install(monkeypatch, lambda gb, r, k, sp: 4.95 if (gb, r, k, sp) == (8, 4, 0, (0, 0, 0))
             else (5.0 if (gb, r, k, sp) == (8, 0, 0, (0, 0, 0)) else 7.0))
    S = [FakeSolver()]
    best, best_ms, _ = autotune.tune(S, passes=2, reps=1)
    assert best == autotune.DEFAULT and best_ms == 5.0
