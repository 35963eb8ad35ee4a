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


def state_and_adjoint_rhs(V, T, k):
    """The two right-hand sides of a body: the plane wave e^{ikz} and the adjoint
    source sum_m G(x - x_obs,m), x_obs at distance 5 along +-x and +-z from the
    body's centre (G = e^{ikr}/(4 pi r))."""
    c, _, _, _ = oracle.geometry(V, T)
    pw = inputs.plane_wave(c, k)
    centre = 0.5 * (V.min(axis=0) + V.max(axis=0))
    adj = np.zeros(c.shape[0], dtype=np.complex128)
    for o in ((5, 0, 0), (-5, 0, 0), (0, 0, 5), (0, 0, -5)):
        r = np.linalg.norm(c - (centre + np.array(o, float)), axis=1)
        adj += np.exp(1j * k * r) / (4 * np.pi * r)
    return np.stack([pw, adj])


def test_batch_solve_state_and_adjoint(cuda_ok):
    """GMRES on every body of a batch at once (two right-hand sides each): per
    system the recursive residual reaches tol, the solution agrees with the
    single-body solve, and the oracle's true residual on 300 rows per body is
    at the apply accuracy."""
    probs = small_bodies()
    batch = Batch(probs, p=10, mode="mixed", max_nrhs=2)
    b = np.concatenate([state_and_adjoint_rhs(V, T, k) for V, T, k in probs], axis=1)
    tol = 1e-8
    x, iters, relres = batch.solve(torch.from_numpy(b).cuda(), tol=tol, max_iter=200, restart=200)
    x = x.cpu().numpy()
    assert relres.shape == (2, len(probs)) and np.all(relres <= tol) and iters >= 2
    # the host-driven loop reaches the same solutions (applies agree to FP32 rounding)
    xh, ih, rh = batch.solve(torch.from_numpy(b).cuda(), tol=tol, max_iter=200, restart=200, driver="host")
    assert abs(ih - iters) <= 1 and np.all(rh <= tol)
    assert rel(x, xh.cpu().numpy()) <= 1e-5
    for p, (V, T, k) in enumerate(probs):
        a, e = batch.offsets[p], batch.offsets[p + 1]
        op = Operator(V, T, k, p=10, mode="mixed", max_nrhs=2)
        xs, _, _ = op.solve(torch.from_numpy(b[:, a:e].copy()).cuda(), tol=tol)
        assert rel(x[:, a:e], xs.cpu().numpy()) <= 1e-5
        rows = np.sort(np.random.default_rng(p).choice(e - a, min(300, e - a), replace=False))
        res = b[:, a:e][:, rows] - oracle.apply(V, T, k, x=x[:, a:e], rows=rows)
        assert np.linalg.norm(res) / np.linalg.norm(b[:, a:e][:, rows]) <= 1e-5


def test_batch_solve_rejects_bad_arguments(cuda_ok):
    from paper_1606_02383_gb300 import _lib
    batch = Batch(small_bodies()[:2], p=8, mode="mixed", max_nrhs=1)
    b = torch.zeros((3, batch.n), dtype=torch.complex128, device="cuda")
    with pytest.raises(RuntimeError):
        batch.solve(b)  # nrhs above max_nrhs
    rc = batch._lib.bem_gmres_solve_batch(batch._h, 1, _lib.BEM_C128, b.data_ptr(), None, 1e-6, 10, 10, 0, None, None,
                                          None)
    assert rc == _lib.BEM_ERR_INVALID_ARG


def test_uneven_batch_with_per_body_options(cuda_ok):
    """Bodies spanning the batching workload's size spread (2,000 to 20,000
    triangles here, ellipsoids and tori, k in [1, 8]), each with its own
    options (trees, near-field units, K slices as an autotuner would pick
    them), applied together: every body against the oracle on sampled rows,
    and against its own single-problem operator."""
    probs = inputs.batch_bodies(6, seed=3, n_min=2000, n_max=20000)
    sizes = [T.shape[0] for _, T, _ in probs]
    assert min(sizes) < 4000 and max(sizes) > 10000, sizes
    opts = [{"leaf_level": -1, "leaf_target": 32}, {"leaf_level": -2, "leaf_target": 32},
            {"leaf_level": 0, "leaf_target": 48, "p2p_unit": 32}, {"leaf_level": 3, "tc_kslice": 8},
            {"leaf_level": -1, "leaf_target": 24, "p2p_unit": 16}, {"leaf_level": 0, "leaf_target": 64}]
    batch = Batch(probs, p=0, eps=1e-5, mode="mixed", max_nrhs=2, options=opts)
    n = batch.n
    x = inputs.random_density(n, 2, seed=61)
    y = inputs.random_density(n, 2, seed=62)
    z = batch.apply(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()).cpu().numpy()
    for b, ((V, T, k), o) in enumerate(zip(probs, opts)):
        a, e = batch.offsets[b], batch.offsets[b + 1]
        op = Operator(V, T, k, p=0, eps=1e-5, mode="mixed", max_nrhs=2, **o)
        zs = op.apply(torch.from_numpy(x[:, a:e]).cuda(), torch.from_numpy(y[:, a:e]).cuda()).cpu().numpy()
        assert rel(z[:, a:e], zs) <= 1e-6, b
        rows = np.sort(np.random.default_rng(b).choice(e - a, 300, replace=False))
        ref = oracle.apply(V, T, k, x=x[:, a:e], y=y[:, a:e], rows=rows)
        assert rel(z[:, a:e][:, rows], ref) <= 1e-5, (b, sizes[b], o)
        op.close()
    batch.close()
