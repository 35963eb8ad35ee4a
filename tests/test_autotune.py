"""Autotuner over the tree and the tile choices: the selection rule on CPU, the tuned operator on GPU."""
import numpy as np
import pytest

import oracle
from paper_1606_02383_gb300 import inputs
from paper_1606_02383_gb300.autotune import pick


def test_pick_takes_the_fastest():
    assert pick({4: 3.0, 5: 2.0, 6: 2.5}) == 5


def test_pick_keeps_the_preferred_within_tolerance():
    assert pick({4: 2.0, 5: 2.03}, prefer=5) == 5          # 1.5 % slower: noise, keep the rule
    assert pick({4: 2.0, 5: 2.10}, prefer=5) == 4          # 5 % slower: switch
    assert pick({4: 2.0, 5: 2.10}, prefer=7) == 4          # unknown preference is ignored


def test_pick_rejects_empty():
    with pytest.raises(ValueError):
        pick({})


@pytest.mark.gpu
def test_tuned_operator_matches_oracle(cuda_ok):
    """The tuned operator keeps the accuracy of every candidate (orders follow
    eps); checked on 300 oracle rows of a 5,120-triangle sphere at ka = 5."""
    import torch
    from paper_1606_02383_gb300.autotune import tune
    V, T = inputs.icosphere(4)
    n = T.shape[0]
    op, report = tune(V, T, 5.0, eps=1e-5, reps=3, warmup=1)
    assert len(report["ms"]) >= 4
    assert report["gain"] >= 1.0
    chosen = report["chosen"]
    assert set(chosen) == {"leaf_level", "leaf_target", "p2p_unit", "tc_kslice", "tc_pipeline", "p2p_stage"}
    if chosen["leaf_level"] > 0:
        assert op.info("leaf_level") == chosen["leaf_level"] and op.info("adaptive") == 0
    else:
        assert op.info("adaptive") == (0 if chosen["leaf_level"] == 0 else 1)
    x = inputs.random_density(n, 1, seed=81)
    y = inputs.random_density(n, 1, seed=82)
    z = op.apply(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()).cpu().numpy()
    rows = np.sort(np.random.default_rng(3).choice(n, 300, replace=False))
    ref = oracle.apply(V, T, 5.0, x=x, y=y, rows=rows)
    assert np.linalg.norm(z[:, rows] - ref) / np.linalg.norm(ref) <= 1e-5
    op.close()
