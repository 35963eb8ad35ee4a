"""Parity at the full sizes of the measured configurations, in the launch
configuration the bench times (automatic orders, mixed mode, eps 1e-5), on
seeded sampled rows that the oracle computes one by one."""
import numpy as np
import pytest
import torch

import oracle
from paper_1606_02383_gb300 import inputs
from paper_1606_02383_gb300.operator import Operator

pytestmark = pytest.mark.gpu


def _sampled_rel_err(V, T, k, rows=200, seed=0):
    n = T.shape[0]
    x = inputs.random_density(n, 1, seed=seed, stream=0)
    y = inputs.random_density(n, 1, seed=seed, stream=1)
    op = Operator(V, T, k, p=0, eps=1e-5, mode="mixed")
    z = op.apply(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()).cpu().numpy()
    op.close()
    sel = np.sort(np.random.default_rng(seed + 7).choice(n, rows, replace=False))
    ref = oracle.apply(V, T, k, x=x, y=y, rows=sel)
    return float(np.linalg.norm(z[:, sel] - ref) / np.linalg.norm(ref))


def test_headline_sphere_327680_ka20(cuda_ok):
    V, T = inputs.icosphere(7)
    assert T.shape[0] == 327680
    assert _sampled_rel_err(V, T, 20.0) <= 1e-5


def test_large_multibody_983040(cuda_ok):
    V, T = inputs.large_multibody()
    assert T.shape[0] == 983040
    assert _sampled_rel_err(V, T, 20.2, seed=3) <= 1e-5
