"""Autotuner over the octree and the kernels' tile choices.

The expansion orders follow ``eps`` on every level, so every candidate meets
the same accuracy; only the split of the work changes:
  - the tree: a uniform leaf level, or the adaptive tree with its depth chosen
    per level-2 region for a target mean occupancy (leaf_target).  Deeper
    leaves shrink the near field (P2P cost grows with the leaf occupancy) and
    multiply the translation pairs (M2L cost grows with the boxes times P^2);
  - the near field's work unit (p2p_unit targets per warp): smaller units
    balance the grid's tail, larger ones load each source for more targets;
  - the translation jobs' K slice (tc_kslice stages): shorter slices give
    small operators more CTAs at the price of more atomic adds;
  - the translation loop (tc_pipeline: per operator, block-synchronous,
    two warp-specialised stages, persistent) and the near field's source
    staging (p2p_stage): which hides latency best depends on the job sizes.
``tune`` times the candidates with CUDA events on the current stream,
coordinate by coordinate (tree first, then the tile and loop choices), and
keeps the fastest operator.
"""
from __future__ import annotations

import numpy as np
import torch

from . import inputs
from .operator import Operator

DEFAULTS = {"leaf_level": 0, "leaf_target": 48, "p2p_unit": 64, "tc_kslice": 16, "tc_pipeline": 0, "p2p_stage": 0}


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


def _key(cfg):
    return tuple(sorted(cfg.items()))


def tune(vertices, triangles, k, p=0, eps=1e-5, mode="mixed", nrhs=1, spread=1, targets=(24, 32, 48, 64),
         units=(32, 64), kslices=(8, 16), pipelines=(0, 1, 2, 3), stages=(0, 1), reps=5, warmup=2, seed=0,
         **options):
    """Returns ``(operator, report)`` with the fastest candidate for ``nrhs``
    right-hand sides.  Candidates: the default uniform tree (leaf_level 0) and
    uniform trees on its level +- ``spread``, the adaptive tree with its depth
    chosen per region (leaf_level -1) for every leaf target in ``targets``;
    then, for the best tree, every p2p_unit in ``units``, every tc_kslice in
    ``kslices``, every tc_pipeline in ``pipelines`` and every p2p_stage in
    ``stages`` (mixed mode only for the last two).  ``report`` holds
    ``{"default": cfg, "chosen": cfg, "ms": [(cfg, ms), ...], "gain": default_ms / chosen_ms}``."""
    n = np.asarray(triangles).shape[0]
    x = torch.from_numpy(inputs.random_density(n, nrhs, seed=seed, stream=0)).cuda()
    y = torch.from_numpy(inputs.random_density(n, nrhs, seed=seed, stream=1)).cuda()
    timed = {}
    state = {"best": None, "best_cfg": None}

    def run(cfg):
        key = _key(cfg)
        if key in timed:
            return timed[key]
        op = Operator(vertices, triangles, k, p=p, eps=eps, mode=mode, max_nrhs=max(nrhs, options.get("max_nrhs", 1)),
                      **{kk: v for kk, v in options.items() if kk != "max_nrhs"}, **cfg)
        timed[key] = _time_apply(op, x, y, reps, warmup)
        if state["best"] is None or pick({0: timed[_key(state["best_cfg"])], 1: timed[key]}, prefer=0) == 1:
            if state["best"] is not None:
                state["best"].close()
            state["best"], state["best_cfg"] = op, dict(cfg)
        else:
            op.close()
        return timed[key]

    default = dict(DEFAULTS)
    run(default)
    deepest = state["best"].info("leaf_level")
    trees = [dict(default, leaf_level=lvl) for lvl in range(deepest - spread, deepest + spread + 1) if 2 <= lvl <= 10]
    trees += [dict(default, leaf_level=-1, leaf_target=t) for t in targets]
    for cfg in trees:
        run(cfg)
    base = dict(state["best_cfg"])
    for u in units:
        run(dict(base, p2p_unit=u))
    base = dict(state["best_cfg"])
    for ks in kslices:
        run(dict(base, tc_kslice=ks))
    if mode == "mixed":
        base = dict(state["best_cfg"])
        for pl in pipelines:
            run(dict(base, tc_pipeline=pl))
        base = dict(state["best_cfg"])
        for st in stages:
            run(dict(base, p2p_stage=st))
    chosen = state["best_cfg"]
    report = {"default": default, "chosen": chosen,
              "ms": [(dict(kk), v) for kk, v in timed.items()],
              "gain": timed[_key(default)] / timed[_key(chosen)]}
    return state["best"], report


def tune_options(vertices, triangles, k, **kw):
    """The tuned option dict alone (the operator is released), e.g. for a
    batch built with per-problem options."""
    op, report = tune(vertices, triangles, k, **kw)
    op.close()
    return report["chosen"], report
