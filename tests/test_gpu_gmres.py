"""GMRES on the device vs the oracle's dense LU and vs the Mie series."""
import numpy as np
import pytest
import torch

import oracle
from oracle import closed_forms as cf
from paper_1606_02383_gb300 import inputs
from paper_1606_02383_gb300.operator import Operator

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode,p,tol_lu", [("direct64", 0, 1e-7), ("mixed", 10, 1e-5)])
def test_gmres_plane_wave_small_sphere(cuda_ok, mode, p, tol_lu):
    """Config 'plain method, small': (1/2 I - D) p = exp(i k z), tol 1e-8, checked against LU and Mie."""
    V, T = inputs.icosphere(3)
    k = 1.0
    c, _, _, _ = oracle.geometry(V, T)
    b = inputs.plane_wave(c, k)[None, :]
    S, D = oracle.assemble(V, T, k)
    ref = oracle.lu_solve(0.5 * np.eye(T.shape[0]) - D, b)
    op = Operator(V, T, k, p=p, mode=mode, leaf_level=3 if mode == "mixed" else 0)
    x, iters, relres = op.solve(torch.from_numpy(b).cuda(), tol=1e-8, max_iter=100, restart=100)
    x = x.cpu().numpy()
    assert relres[0] <= 1e-8
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= tol_lu
    mie = cf.mie_rigid_sphere_surface(k, 1.0, c[:, 2] / np.linalg.norm(c, axis=1))
    assert np.linalg.norm(x[0] - mie) / np.linalg.norm(mie) <= 5e-3
    assert 2 <= iters <= 40


def test_gmres_multi_rhs_and_restart(cuda_ok):
    V, T = inputs.icosphere(3)
    k = 2.0
    n = T.shape[0]
    rng = np.random.default_rng(0)
    b = inputs.random_density(n, 3, seed=4)
    op = Operator(V, T, k, mode="direct64")
    x, iters, relres = op.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_iter=300, restart=7)
    assert np.all(relres <= 1e-10)
    Ax = op.apply(x, None).cpu().numpy()
    assert np.linalg.norm(Ax - b) / np.linalg.norm(b) <= 1e-9
    del rng


def test_gmres_not_converged_status(cuda_ok):
    from paper_1606_02383_gb300 import _lib
    V, T = inputs.icosphere(2)
    op = Operator(V, T, 1.0, mode="direct64")
    b = torch.from_numpy(inputs.random_density(T.shape[0], 1, seed=2)).cuda()
    with pytest.raises(_lib.BemError) as e:
        op.solve(b, tol=1e-14, max_iter=2, restart=2)
    assert e.value.code == _lib.BEM_ERR_NOT_CONVERGED
    x, iters, rel = op.solve(b, tol=1e-14, max_iter=2, restart=2, raise_on_fail=False)
    assert iters == 2 and rel[0] > 1e-14


def test_state_and_adjoint_rhs_in_one_solve(cuda_ok):
    """State (plane wave) and adjoint (point sources at the observation points,
    Section 2.2: same matrix, right-hand side sum_m G(x - x_obs,m)) solved
    together as nrhs = 2, each checked against the oracle's LU solve."""
    V, T = inputs.icosphere(3)
    k = 2.0
    c, _, _, _ = oracle.geometry(V, T)
    obs = np.array([[5.0, 0, 0], [-5.0, 0, 0], [0, 0, 5.0], [0, 0, -5.0]])
    r = np.linalg.norm(c[:, None, :] - obs[None, :, :], axis=2)
    adj = np.sum(np.exp(1j * k * r) / (4 * np.pi * r), axis=1)
    b = np.stack([inputs.plane_wave(c, k), adj])
    S, D = oracle.assemble(V, T, k)
    ref = oracle.lu_solve(0.5 * np.eye(T.shape[0]) - D, b)
    op = Operator(V, T, k, p=10, mode="mixed", leaf_level=3)
    x, iters, relres = op.solve(torch.from_numpy(b).cuda(), tol=1e-8, max_iter=100, restart=100)
    x = x.cpu().numpy()
    assert np.all(relres <= 1e-8)
    for q in range(2):
        assert np.linalg.norm(x[q] - ref[q]) / np.linalg.norm(ref[q]) <= 1e-5


@pytest.mark.parametrize("mode,restart", [("direct64", 7), ("direct64", 300), ("mixed", 9)])
def test_graph_cycles_match_host_loop(cuda_ok, mode, restart):
    """The graph-resident cycles (Arnoldi steps in a conditional WHILE node,
    Givens rotations on the device) reach the same iterates as the host-driven
    loop: same iteration count, the same solution to rounding, and residuals
    that agree with the operator's own A x - b.  Three right-hand sides of
    different difficulty converge at different steps, and restart = 7 or 9
    makes several cycles."""
    V, T = inputs.icosphere(3)
    k = 2.0
    n = T.shape[0]
    c, _, _, _ = oracle.geometry(V, T)
    b = np.concatenate([inputs.random_density(n, 2, seed=8), inputs.plane_wave(c, k)[None, :]])
    op = Operator(V, T, k, p=10, mode=mode, leaf_level=0 if mode == "direct64" else 3, max_nrhs=3)
    bd = torch.from_numpy(b).cuda()
    tol = 1e-10 if mode == "direct64" else 1e-6
    xg, ig, rg = op.solve(bd, tol=tol, max_iter=300, restart=restart, driver="graph_only")
    xh, ih, rh = op.solve(bd, tol=tol, max_iter=300, restart=restart, driver="host")
    xg, xh = xg.cpu().numpy(), xh.cpu().numpy()
    assert np.all(rg <= tol) and np.all(rh <= tol)
    if mode == "direct64":  # deterministic applies: the two drivers differ only in the Givens rounding
        assert ig == ih
        assert np.allclose(rg, rh, rtol=1e-6, atol=1e-3 * tol)
        assert np.linalg.norm(xg - xh) / np.linalg.norm(xh) <= 1e-9
    else:  # the tensor-core epilogue adds with float atomics: applies agree to FP32 rounding
        assert abs(ig - ih) <= 1
        assert np.linalg.norm(xg - xh) / np.linalg.norm(xh) <= 1e-5
    true = np.linalg.norm(op.apply(torch.from_numpy(xg).cuda(), None).cpu().numpy() - b, axis=1) / np.linalg.norm(b, axis=1)
    assert np.all(true <= 10 * tol)


def test_graph_cycles_max_iter_and_zero_rhs(cuda_ok):
    """The device loop stops at max_iter (mid-cycle) with BEM_ERR_NOT_CONVERGED,
    and a zero right-hand side converges at once with x = 0."""
    from paper_1606_02383_gb300 import _lib
    V, T = inputs.icosphere(2)
    n = T.shape[0]
    op = Operator(V, T, 1.0, mode="direct64", max_nrhs=2)
    b = torch.from_numpy(inputs.random_density(n, 1, seed=2)).cuda()
    x, iters, rel = op.solve(b, tol=1e-14, max_iter=5, restart=3, raise_on_fail=False, driver="graph_only")
    xh, ih, relh = op.solve(b, tol=1e-14, max_iter=5, restart=3, raise_on_fail=False, driver="host")
    assert iters == ih == 5 and rel[0] > 1e-14
    assert np.isclose(rel[0], relh[0], rtol=1e-6)
    with pytest.raises(_lib.BemError) as e:
        op.solve(b, tol=1e-14, max_iter=5, restart=3, driver="graph_only")
    assert e.value.code == _lib.BEM_ERR_NOT_CONVERGED
    b2 = torch.zeros((2, n), dtype=torch.complex128, device="cuda")
    b2[1] = b[0]
    x2, it2, rel2 = op.solve(b2, tol=1e-10, max_iter=100, driver="graph_only")
    assert rel2[0] == 0.0 and rel2[1] <= 1e-10
    assert torch.count_nonzero(x2[0]).item() == 0
