"""Autotuner over the octree's leaf level (the leaf size of the FMM).

The expansion orders follow ``eps`` at every level, so every candidate meets
the same accuracy. Only the split of the work changes: a deeper leaf level
shrinks the near field (P2P cost grows with the leaf occupancy) and multiplies
the translation pairs (M2L cost grows with the number of boxes times P^2).
``tune`` builds the operator at the rule-based leaf level and at its
neighbours, times applies of each with CUDA events on the current stream, and
keeps the fastest.
"""
from __future__ import annotations

import numpy as np
import torch

from . import inputs
from .operator import Operator


def pick(timings: dict, prefer=None, tolerance: float = 0.02):
    """The fastest key of ``{key: milliseconds}``. ``prefer`` (e.g. the rule-based
    choice) wins whenever it is within ``tolerance`` of the fastest, so that
    timing noise does not move the choice."""
    if not timings:
        raise ValueError("no timings")
    best = min(timings, key=lambda key: timings[key])
    if prefer is not None and prefer in timings and timings[prefer] <= timings[best] * (1.0 + tolerance):
        return prefer
    return best


def _time_apply(op: Operator, x, y, reps: int, warmup: int) -> float:
    for _ in range(warmup):
        op.apply(x, y)
    stream = torch.cuda.current_stream()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(reps):
        op.apply(x, y)
    t1.record(stream)
    t1.synchronize()
    return t0.elapsed_time(t1) / reps


def tune(vertices, triangles, k, p=0, eps=1e-5, mode="mixed", nrhs=1, spread=1, reps=5, warmup=2, seed=0,
         **options):
    """Returns ``(operator, report)``: the fastest of the leaf levels L0 - spread
    .. L0 + spread (L0 the rule-based level, levels 2..10) for ``nrhs``
    right-hand sides, and ``report = {"rule": L0, "chosen": L, "ms": {L: ms}}``.
    The operators that lose are destroyed as soon as they are timed."""
    n = np.asarray(triangles).shape[0]
    x = torch.from_numpy(inputs.random_density(n, nrhs, seed=seed, stream=0)).cuda()
    y = torch.from_numpy(inputs.random_density(n, nrhs, seed=seed, stream=1)).cuda()
    best = Operator(vertices, triangles, k, p=p, eps=eps, mode=mode, **options)
    rule = best.info("leaf_level")
    ms = {rule: _time_apply(best, x, y, reps, warmup)}
    best_level = rule
    for level in range(rule - spread, rule + spread + 1):
        if level == rule or level < 2 or level > 10:
            continue
        op = Operator(vertices, triangles, k, p=p, eps=eps, mode=mode, leaf_level=level, **options)
        ms[level] = _time_apply(op, x, y, reps, warmup)
        if pick({best_level: ms[best_level], level: ms[level]}, prefer=best_level) == level:
            best.close()
            best, best_level = op, level
        else:
            op.close()
    chosen = pick(ms, prefer=rule)
    if chosen != best_level:
        # the rule-based level lost by less than the tolerance to a level already closed
        best.close()
        best = Operator(vertices, triangles, k, p=p, eps=eps, mode=mode, leaf_level=chosen, **options)
    return best, {"rule": rule, "chosen": chosen, "ms": ms}
