"""Batches of independent scatterers (ellipsoids and tori, own wavenumbers)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1606_02383_gb300 import inputs
from paper_1606_02383_gb300.operator import Batch, Operator

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def small_bodies():
    return [(*inputs.ellipsoid(6, (1.0, 0.7, 1.4)), 1.5), (*inputs.torus(30, 10, 1.0, 0.3), 3.0),
            (*inputs.ellipsoid(9, (0.6, 1.2, 0.9)), 5.0), (*inputs.torus(40, 12, 1.0, 0.45), 2.2),
            (*inputs.icosphere(3, 0.8), 4.0), (*inputs.ellipsoid(4, (2.0, 0.5, 0.8)), 7.5)]


@pytest.mark.parametrize("nrhs", [1, 2])
def test_batch_matches_single_problem_applies_and_oracle(cuda_ok, nrhs):
    probs = small_bodies()
    batch = Batch(probs, p=10, mode="mixed", max_nrhs=2)
    n = batch.n
    x = inputs.random_density(n, nrhs, seed=51)
    y = inputs.random_density(n, nrhs, seed=52)
    for rep in range(2):  # the second call replays the captured graph
        z = batch.apply(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()).cpu().numpy()
        for b, (V, T, k) in enumerate(probs):
            a, e = batch.offsets[b], batch.offsets[b + 1]
            op = Operator(V, T, k, p=10, mode="mixed", max_nrhs=2)
            zs = op.apply(torch.from_numpy(x[:, a:e]).cuda(), torch.from_numpy(y[:, a:e]).cuda()).cpu().numpy()
            assert rel(z[:, a:e], zs) <= 1e-6
            ref = oracle.apply(V, T, k, x=x[:, a:e], y=y[:, a:e])
            assert rel(z[:, a:e], ref) <= 1e-5


def test_batch_generators_are_closed_surfaces():
    for V, T, k in inputs.batch_bodies(6, seed=1, n_min=300, n_max=3000):
        c, area, nrm, _ = oracle.geometry(V, T)
        assert np.max(np.abs((area[:, None] * nrm).sum(0))) < 1e-12
        assert 1.0 <= k <= 8.0
