"""dL/dk (bem_grad) against central finite differences of the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1606_02383_gb300 import inputs
from paper_1606_02383_gb300.operator import Operator

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("mode,p,leaf", [("direct64", 0, 0), ("mixed", 10, 3)])
@pytest.mark.parametrize("k", [1.0, 4.0])
def test_dk_matches_oracle_central_difference(cuda_ok, mode, p, leaf, k):
    V, T = inputs.icosphere(3)
    n = T.shape[0]
    x = inputs.random_density(n, 1, seed=31)
    y = inputs.random_density(n, 1, seed=32)
    g = inputs.random_density(n, 1, seed=33)
    h = 1e-6

    def loss(kk):
        return float(np.real(np.vdot(g, oracle.apply(V, T, kk, x=x, y=y))))

    fd = (loss(k + h) - loss(k - h)) / (2 * h)
    op = Operator(V, T, k, p=p, mode=mode, leaf_level=leaf)
    dk = op.grad_k(dev(g), dev(x), dev(y))
    assert abs(dk - fd) <= 1e-6 * abs(fd)


def test_dk_single_layer_only_and_autograd(cuda_ok):
    V, T = inputs.icosphere(2)
    n = T.shape[0]
    k = 2.5
    y = inputs.random_density(n, 1, seed=41)
    t = inputs.random_density(n, 1, seed=42)
    h = 1e-6

    def loss(kk):
        z = oracle.apply(V, T, kk, y=y)
        return float(np.sum(np.abs(z - t) ** 2))

    fd = (loss(k + h) - loss(k - h)) / (2 * h)
    op = Operator(V, T, k, mode="direct64")
    kt = torch.tensor(k, dtype=torch.float64, requires_grad=True)
    yt = dev(y).requires_grad_(True)
    xt = torch.zeros_like(yt)
    L = (op(xt, yt, kt) - dev(t)).abs().pow(2).sum()
    L.backward()
    assert abs(float(kt.grad) - fd) <= 1e-6 * abs(fd)
