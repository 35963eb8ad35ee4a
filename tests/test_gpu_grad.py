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


# --- vertex gradients -------------------------------------------------------

def _jittered(level, seed=3, amp=0.05):
    V, T = inputs.icosphere(level)
    rng = np.random.default_rng(seed)
    return V * (1.0 + amp * rng.standard_normal((V.shape[0], 1))), T


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("mesh", ["icosphere3_jittered", "level_set_slivers"])
@pytest.mark.parametrize("mode,p,leaf,direct,tol", [("direct64", 0, 0, 0, 1e-10), ("mixed", 10, 3, 1, 1e-5),
                                                    ("mixed", 10, 3, 0, 1e-4), ("fp64", 16, 3, 0, 2e-6)])
def test_vertex_gradient_matches_oracle(cuda_ok, mesh, mode, p, leaf, direct, tol):
    """Every vertex: GPU dL/dV against the oracle's dual-number gradient.  FP64
    direct differs only by rounding.  With direct = 1 the mixed mode sums the
    regular rule over all pairs in FP32 (block-relative coordinates split into
    high and low parts, FP64 between tiles) and keeps the corrections in FP64,
    which gives about 1e-6.  Through the tree (direct = 0) the far boxes add the
    truncation of their expansions, first and second derivatives included:
    measured 2e-5 (mixed, p = 10) and 1e-6 (FP64, p = 16) on the jittered
    sphere, whose leaves are only about 1.5 longest edges wide."""
    if mesh == "icosphere3_jittered":
        V, T = _jittered(3)
    else:
        V, T = inputs.level_set_mesh(seed=4, grid=24, target=1200)
    n = T.shape[0]
    k = 2.7
    x, y, g = (inputs.random_density(n, 2, seed=s) for s in (51, 52, 53))
    dV_ref, dk_ref = oracle.grad(V, T, k, g, x, y)
    op = Operator(V, T, k, p=p, mode=mode, leaf_level=leaf, grad_direct=direct)
    dV, dk = op.grad(dev(g), dev(x), dev(y))
    assert _rel(dV, dV_ref) <= tol, _rel(dV, dV_ref)
    assert abs(dk - dk_ref) <= max(tol, 1e-9) * abs(dk_ref)


@pytest.mark.parametrize("direct,tol", [(1, 1e-5), (0, 1e-4)])
def test_vertex_gradient_sampled_at_30k(cuda_ok, direct, tol):
    """The 30,000-triangle level-set surface of the differentiation workload
    (k = 3, mixed FMM, orders from eps = 1e-5): sampled vertices against the
    oracle, which differentiates only the pairs that touch them.  Through the
    tree (direct = 0) the far boxes' expansions, differentiated twice, add
    their truncation (measured 3e-5 on these vertices)."""
    V, T = inputs.level_set_mesh(seed=0)
    n = T.shape[0]
    k = 3.0
    x, y, g = (inputs.random_density(n, 1, seed=s) for s in (61, 62, 63))
    op = Operator(V, T, k, mode="mixed", grad_direct=direct)
    dV, dk = op.grad(dev(g), dev(x), dev(y), k=False)
    assert dk is None
    rng = np.random.default_rng(7)
    sel = rng.choice(V.shape[0], 6, replace=False)
    ref, _ = oracle.grad(V, T, k, g, x, y, vertices=sel)
    assert _rel(dV[sel], ref) <= tol, _rel(dV[sel], ref)


@pytest.mark.parametrize("mode,p,leaf,tol", [("mixed", 12, -2, 3e-5), ("mixed", 12, -1, 3e-5),
                                           ("fp64", 18, -2, 3e-8)])
def test_vertex_gradient_tree_against_all_pairs(cuda_ok, mode, p, leaf, tol):
    """The tree's regular-rule sums against the all-pairs sums of the same
    handle (grad_direct = 1), on adaptive trees with five right-hand sides
    (the far and near passes in chunks of 4 and 1); dL/dk is unaffected."""
    V1, T1 = inputs.icosphere(3)
    V2, T2 = inputs.icosphere(3, 0.3, (1.3, 0.4, -0.2))
    V, T = inputs.merge_meshes([(V1, T1), (V2, T2)])
    n = T.shape[0]
    k = 3.3
    x, y, g = (inputs.random_density(n, 5, seed=s) for s in (81, 82, 83))
    common = dict(p=p, mode=mode, leaf_level=leaf, leaf_target=16, max_nrhs=5)
    op = Operator(V, T, k, **common)
    levels = {l for l in range(11) if op.info(200 + l) > 0}
    assert len(levels) >= 2, levels
    ref = Operator(V, T, k, grad_direct=1, **common)
    dV, dk = op.grad(dev(g), dev(x), dev(y))
    dV_ref, dk_ref = ref.grad(dev(g), dev(x), dev(y))
    assert _rel(dV, dV_ref) <= tol, _rel(dV, dV_ref)
    assert abs(dk - dk_ref) <= 1e-6 * abs(dk_ref)
    op.close()
    ref.close()


def test_vertex_gradient_autograd(cuda_ok):
    """L = sum |z - t|^2 through torch.autograd; the upstream gradient is 2 (z - t)."""
    V, T = _jittered(2, seed=9)
    n = T.shape[0]
    k = 1.9
    x, y, t = (inputs.random_density(n, 1, seed=s) for s in (71, 72, 73))
    op = Operator(V, T, k, mode="direct64")
    Vt = torch.from_numpy(V.copy()).requires_grad_(True)
    L = (op(dev(x), dev(y), vertices=Vt) - dev(t)).abs().pow(2).sum()
    L.backward()
    z = oracle.apply(V, T, k, x=x, y=y)
    ref, _ = oracle.grad(V, T, k, 2.0 * (z - t), x, y)
    assert _rel(Vt.grad.numpy(), ref) <= 1e-10


def test_vertex_gradient_rejects_device_output(cuda_ok):
    import ctypes
    from paper_1606_02383_gb300 import _lib
    V, T = inputs.icosphere(1)
    op = Operator(V, T, 1.0, mode="direct64")
    g = dev(inputs.random_density(T.shape[0], 1, seed=1))
    out = torch.zeros(V.shape[0] * 3, dtype=torch.float64, device="cuda")
    rc = op._lib.bem_grad(op._h, 1, _lib.BEM_C128, g.data_ptr(), None, g.data_ptr(),
                          ctypes.cast(out.data_ptr(), ctypes.POINTER(ctypes.c_double)), None, None)
    assert rc == _lib.BEM_ERR_INVALID_ARG
