"""Autotuner for batched solves of many uneven instances.

A batched solve (maxflow_solve_batched) runs every instance in one persistent
launch, groups of CTAs taking instances from a queue.  Its speed depends on
knobs that have no single best value across graph families: CTAs per group,
discharge rounds and KERNEL_CYCLES per instance, and the work-split
thresholds (rows handled by one thread / one warp / one CTA in the
discharge, rows split into work items in the BFS).  The tuner measures static
batched solves (their state is reset by the solve itself, so every trial
starts from the same point) and does coordinate descent over the knobs.
Single trials are noisy (a batched solve varies by several percent from run to
run), so a trial must beat the best so far by MARGIN to replace it, and a
result other than the default must beat it again in a final interleaved
comparison, or the default stays.
"""
from __future__ import annotations

from . import native

GROUP_BLOCKS = (1, 2, 4, 8, 16, 32)
ROUNDS = (0, 1, 4, 16, 64)            # 0: the adaptive count
CYCLES = (0, 4, 16)                   # 0: the average-degree heuristic
# (0, 0, 0): each instance's own default split (thread rows of 4 or 8 slots by its average degree)
SPLITS = ((0, 0, 0), (8, 512, 256), (4, 256, 128), (16, 2048, 1024), (32, 8192, 4096))
DEFAULT = {"group_blocks": 8, "rounds": 0, "cycles": 0, "split": (0, 0, 0)}
MARGIN = 0.02                         # the fraction a trial must win by


def apply_config(solvers, cfg):
    for s in solvers:
        s.set_rounds(cfg["rounds"])
        s.set_kernel_cycles(cfg["cycles"])
        s.set_tuning(*cfg["split"])


def measure(solvers, cfg, reps=2):
    apply_config(solvers, cfg)
    return min(native.maxflow_solve_batched(solvers, None, group_blocks=cfg["group_blocks"]) for _ in range(reps))


def tune(solvers, passes=2, reps=2, confirm_reps=5, log=None):
    """Coordinate descent from DEFAULT, then the confirmation against DEFAULT;
    returns (chosen config, its ms, trial log)."""
    best = dict(DEFAULT)
    best_ms = measure(solvers, best, reps)
    trials = [(dict(best), best_ms)]
    space = {"group_blocks": GROUP_BLOCKS, "rounds": ROUNDS, "cycles": CYCLES, "split": SPLITS}
    for _ in range(passes):
        improved = False
        for key, values in space.items():
            for v in values:
                if v == best[key]:
                    continue
                cfg = dict(best)
                cfg[key] = v
                ms = measure(solvers, cfg, reps)
                trials.append((cfg, ms))
                if log:
                    log(f"  {key}={v}: {ms:.3f} ms (best {best_ms:.3f})")
                if ms < best_ms * (1.0 - MARGIN):
                    best, best_ms, improved = cfg, ms, True
        if not improved:
            break
    if best != DEFAULT:
        t_best, t_def = [], []
        for _ in range(confirm_reps):
            t_best.append(measure(solvers, best, 1))
            t_def.append(measure(solvers, DEFAULT, 1))
        if log:
            log(f"  confirm: best {min(t_best):.3f} ms, default {min(t_def):.3f} ms")
        if min(t_best) < min(t_def) * (1.0 - MARGIN):
            best_ms = min(t_best)
        else:
            best, best_ms = dict(DEFAULT), min(t_def)
    apply_config(solvers, best)
    return best, best_ms, trials
