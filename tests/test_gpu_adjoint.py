"""Conjugate-transpose apply (bem_apply_adjoint) and the autograd wrapper."""
import numpy as np
import pytest
import torch

import oracle
from paper_1606_02383_gb300 import inputs
from paper_1606_02383_gb300.operator import Operator

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("mode,p,leaf,tol", [("direct64", 0, 0, 1e-10), ("fp64", 10, 3, 1e-5), ("mixed", 10, 3, 1e-5),
                                             ("mixed", 0, 0, 1e-5)])
def test_adjoint_matches_oracle(cuda_ok, mode, p, leaf, tol):
    V, T = inputs.icosphere(3)
    n = T.shape[0]
    k = 2.0
    g = inputs.random_density(n, 2, seed=21)
    gx_ref, gy_ref = oracle.adjoint(V, T, k, g)
    op = Operator(V, T, k, p=p, mode=mode, leaf_level=leaf)
    gx, gy = op.adjoint(dev(g))
    assert rel(gx.cpu().numpy(), gx_ref) <= tol
    assert rel(gy.cpu().numpy(), gy_ref) <= tol


@pytest.mark.parametrize("mode,p,leaf,tol", [("direct64", 0, 0, 1e-12), ("fp64", 10, 3, 1e-12), ("mixed", 10, 3, 1e-6)])
def test_dot_product_identity(cuda_ok, mode, p, leaf, tol):
    """<A u, g> = <u, A^H g>: the adjoint is the exact transpose of the discrete
    operator (FMM included), so this holds to rounding."""
    V, T = inputs.icosphere(4)
    n = T.shape[0]
    k = 3.0
    op = Operator(V, T, k, p=p, mode=mode, leaf_level=leaf)
    x = inputs.random_density(n, 1, seed=1)
    y = inputs.random_density(n, 1, seed=2)
    g = inputs.random_density(n, 1, seed=3)
    z = op.apply(dev(x), dev(y)).cpu().numpy()
    gx, gy = op.adjoint(dev(g))
    lhs = np.vdot(g, z)
    rhs = np.vdot(gx.cpu().numpy(), x) + np.vdot(gy.cpu().numpy(), y)
    assert abs(lhs - rhs) <= tol * np.linalg.norm(z) * np.linalg.norm(g)


def test_autograd_gradcheck(cuda_ok):
    """Gradients of a real loss through the operator vs central finite differences."""
    V, T = inputs.icosphere(1)
    n = T.shape[0]
    op = Operator(V, T, 1.5, mode="direct64")
    x = dev(inputs.random_density(n, 1, seed=5)).requires_grad_(True)
    y = dev(inputs.random_density(n, 1, seed=6)).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda a, b: op(a, b), (x, y), eps=1e-6, atol=1e-7, rtol=1e-6)


def test_autograd_matches_oracle_gradient(cuda_ok):
    """dL/dx, dL/dy of L = sum |z - t|^2 vs the oracle's explicit A^H."""
    V, T = inputs.icosphere(3)
    n = T.shape[0]
    k = 2.0
    x = inputs.random_density(n, 1, seed=7)
    y = inputs.random_density(n, 1, seed=8)
    t = inputs.random_density(n, 1, seed=9)
    op = Operator(V, T, k, p=10, mode="mixed", leaf_level=3)
    xt, yt = dev(x).requires_grad_(True), dev(y).requires_grad_(True)
    loss = (op(xt, yt) - dev(t)).abs().pow(2).sum()
    loss.backward()
    # dL/d conj(z) convention: grad_z = 2 (z - t); grad_u = A^H grad_z
    z = oracle.apply(V, T, k, x=x, y=y)
    gx_ref, gy_ref = oracle.adjoint(V, T, k, 2.0 * (z - t))
    assert rel(xt.grad.cpu().numpy(), gx_ref) <= 1e-5
    assert rel(yt.grad.cpu().numpy(), gy_ref) <= 1e-5
