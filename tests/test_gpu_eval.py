"""Field at off-surface points (bem_eval_points) vs the oracle's eval_points.

The points are a lattice in its natural order around the sphere, points on
rays just off the surface (between 0.3 and 6 longest edges away, so every
rule R_0, R_1, R_2 is used), points 50 radii away (outside the tree's root
cube) and the centre (in an empty box).  Tolerances: the direct sums as the
apply, 1e-10 relative L2 in the FP64 modes (same rules, only rounding
differs) and 1e-5 in the mixed mode; the FMM walk (multipoles of far boxes)
1e-5 in the mixed mode and 1e-8 in the FP64 mode at order 16, where the
truncation measured 1e-9 (1.6e-10 with leaves on level 2).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1606_02383_gb300 import _lib, inputs
from paper_1606_02383_gb300.operator import Operator

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def field_points(V, T):
    g = np.linspace(-1.9, 1.9, 9)
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    lat = lat[np.abs(np.linalg.norm(lat, axis=1) - 1.0) > 0.12]
    c, _, _, _ = oracle.geometry(V, T)
    h = np.max(np.linalg.norm(V[T[:, 1]] - V[T[:, 0]], axis=1))
    rng = np.random.default_rng(4)
    idx = rng.choice(T.shape[0], 120, replace=False)
    dirs = c[idx] / np.linalg.norm(c[idx], axis=1, keepdims=True)
    off = h * np.geomspace(0.3, 6.0, 120) * np.where(np.arange(120) % 2 == 0, 1.0, -1.0)
    near = c[idx] + dirs * off[:, None]
    order = np.argsort(np.arctan2(near[:, 1], near[:, 0]))  # neighbours along a curve
    far = rng.normal(size=(20, 3))
    far = 50.0 * far / np.linalg.norm(far, axis=1, keepdims=True)
    return np.concatenate([lat, near[order], far, np.zeros((1, 3))])


# (mode, direct sum, order, tolerance)
EVAL_CASES = [("direct64", False, 10, 1e-10), ("fp64", True, 10, 1e-10), ("mixed", True, 10, 1e-5),
              ("fp64", False, 16, 1e-8), ("mixed", False, 10, 1e-5)]


@pytest.mark.parametrize("mode,direct,p,tol", EVAL_CASES)
def test_eval_points_matches_oracle(cuda_ok, mode, direct, p, tol):
    V, T = inputs.icosphere(3)
    n, k = T.shape[0], 2.0
    x = inputs.random_density(n, 2, seed=9, stream=0)
    y = inputs.random_density(n, 2, seed=9, stream=1)
    pts = field_points(V, T)
    ref = oracle.eval_points(V, T, k, pts, x=x, y=y)
    op = Operator(V, T, k, p=p, mode=mode, leaf_level=0 if mode == "direct64" else 3, max_nrhs=2)
    u = op.eval_points(pts, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), direct=direct).cpu().numpy()
    assert u.shape == ref.shape
    assert rel(u, ref) <= tol
    # each layer alone, and single precision output
    us = op.eval_points(pts, None, torch.from_numpy(y).cuda(), direct=direct).cpu().numpy()
    assert rel(us, oracle.eval_points(V, T, k, pts, y=y)) <= tol
    u64 = op.eval_points(pts, torch.from_numpy(x.astype(np.complex64)).cuda(),
                         torch.from_numpy(y.astype(np.complex64)).cuda(), direct=direct).cpu().numpy()
    assert u64.dtype == np.complex64 and rel(u64, ref) <= max(tol, 2e-6)
    op.close()


@pytest.mark.parametrize("mode,direct,p,tol", EVAL_CASES)
def test_eval_points_gradient_matches_oracle(cuda_ok, mode, direct, p, tol):
    """grad u at the same points (every rule used) against the oracle's
    gradient; the value-and-gradient layout holds the same numbers."""
    V, T = inputs.icosphere(3)
    n, k = T.shape[0], 2.0
    x = inputs.random_density(n, 2, seed=10, stream=0)
    y = inputs.random_density(n, 2, seed=10, stream=1)
    pts = field_points(V, T)
    ref = oracle.eval_points_grad(V, T, k, pts, x=x, y=y)
    op = Operator(V, T, k, p=p, mode=mode, leaf_level=0 if mode == "direct64" else 3, max_nrhs=2)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    g = op.eval_points(pts, xd, yd, gradient=True, direct=direct).cpu().numpy()
    assert g.shape == ref.shape
    assert rel(g, ref) <= tol
    u = op.eval_points(pts, xd, yd, direct=direct).cpu().numpy()
    ug = op.eval_points(pts, xd, yd, value_and_gradient=True, direct=direct).cpu().numpy()
    assert ug.shape == (2, pts.shape[0], 4)
    # the same sums (FP32 contraction may differ between the kernels' variants)
    assert rel(ug[..., 0], u) <= 1e-6 and rel(ug[..., 1:], g) <= 1e-6
    op.close()


def test_eval_points_gauss_identity_and_errors(cuda_ok):
    """At k -> 0 the double layer of a unit density is -1 inside and 0 outside
    (the orientation of Section 2.1's normals); bad arguments are rejected."""
    V, T = inputs.icosphere(3)
    n = T.shape[0]
    op = Operator(V, T, 1e-9, mode="direct64")
    pts = np.array([[0.0, 0.0, 0.0], [0.3, -0.2, 0.1], [2.0, 0.5, 0.0], [0.0, -3.0, 1.0]])
    u = op.eval_points(pts, torch.ones((1, n), dtype=torch.complex128, device="cuda"), None).cpu().numpy()[0]
    # u = -D 1: inside D 1 = -1, outside 0
    assert np.allclose(u[:2], 1.0, atol=2e-3) and np.allclose(u[2:], 0.0, atol=2e-3)
    with pytest.raises(_lib.BemError):
        op.eval_points(np.zeros((0, 3)), torch.ones((1, n), dtype=torch.complex128, device="cuda"))
    op.close()


def test_scattered_field_of_the_solved_rigid_sphere(cuda_ok):
    """End to end: GMRES for the rigid sphere's surface pressure, then the
    scattered field p_s = D p at exterior points through bem_eval_points
    (which returns S y - D x), against the Mie series (discretisation error of
    the 5,120-triangle sphere) and against the oracle's evaluation of the same
    surface solution (1e-5)."""
    from oracle import closed_forms as cf
    V, T = inputs.icosphere(4)
    k = 2.0
    c, _, _, _ = oracle.geometry(V, T)
    op = Operator(V, T, k, p=0, eps=1e-6, mode="mixed")
    b = torch.from_numpy(inputs.plane_wave(c, k)[None, :]).cuda()
    p, iters, relres = op.solve(b, tol=1e-8, max_iter=100, restart=100)
    rng = np.random.default_rng(3)
    d = rng.normal(size=(64, 3))
    pts = d / np.linalg.norm(d, axis=1, keepdims=True) * rng.uniform(1.5, 3.0, size=(64, 1))
    pts = pts[np.argsort(np.arctan2(pts[:, 1], pts[:, 0]))]
    ps = -op.eval_points(pts, x=p).cpu().numpy()[0]
    assert rel(ps, cf.mie_rigid_sphere_scattered(k, 1.0, pts)) < 1e-2
    assert rel(ps, -oracle.eval_points(V, T, k, pts, x=p.cpu().numpy())[0]) < 1e-5
    op.close()


@pytest.mark.parametrize("mode,tol", [("direct64", 1e-7), ("mixed", 1e-5)])
def test_state_observation_adjoint_chain(cuda_ok, mode, tol):
    """Section 2.2's chain for f = 1/2 sum_m |p(x_m)|^2: state solve, the
    pressure at the observers through the representation formula, the
    adjoint right-hand side with weights conj(p(x_m)), the adjoint solve;
    every step against the oracle's dense LU and off-surface evaluation."""
    V, T = inputs.icosphere(3)
    k = 2.0
    c, _, _, _ = oracle.geometry(V, T)
    obs = np.array([[5.0, 0, 0], [-5.0, 0, 0], [0, 0, 5.0], [0, 0, -5.0]])
    b = inputs.plane_wave(c, k)[None, :]
    S, D = oracle.assemble(V, T, k)
    A = 0.5 * np.eye(T.shape[0]) - D
    p_ref = oracle.lu_solve(A, b)
    inc_obs = np.exp(1j * k * obs[:, 2])
    pobs_ref = inc_obs - oracle.eval_points(V, T, k, obs, x=p_ref)[0]
    r = np.linalg.norm(c[:, None, :] - obs[None, :, :], axis=2)
    badj_ref = (np.exp(1j * k * r) / (4 * np.pi * r)) @ np.conj(pobs_ref)
    padj_ref = oracle.lu_solve(A, badj_ref[None, :])
    op = Operator(V, T, k, p=10, mode=mode, leaf_level=0 if mode == "direct64" else 3, max_nrhs=2)
    out = op.state_and_adjoint(torch.from_numpy(b).cuda(), obs, inc_obs, tol=1e-10 if mode == "direct64" else 1e-8)
    assert rel(out["p"].cpu().numpy(), p_ref) <= tol
    assert rel(out["p_obs"].cpu().numpy()[0], pobs_ref) <= tol
    badj = op.point_sources(obs, np.conj(pobs_ref)).cpu().numpy()[0]
    assert rel(badj, badj_ref) <= 1e-12
    assert rel(out["p_adj"].cpu().numpy(), padj_ref) <= tol
    op.close()


@pytest.mark.parametrize("mode,tol", [("direct64", 1e-7), ("mixed", 1e-4)])
def test_topological_derivative_on_a_lattice(cuda_ok, mode, tol):
    """T(x) = Re[3/2 grad p . grad pa - k^2 p pa] (Section 2.5, sound-hard limit)
    on lattice points around the rigid sphere, built from the state and adjoint
    chain, against the same quantity composed from the oracle's LU solutions,
    off-surface values and gradients."""
    V, T = inputs.icosphere(3)
    k = 2.0
    c, _, _, _ = oracle.geometry(V, T)
    obs = np.array([[5.0, 0, 0], [-5.0, 0, 0], [0, 0, 5.0], [0, 0, -5.0]])
    b = inputs.plane_wave(c, k)[None, :]
    S, D = oracle.assemble(V, T, k)
    A = 0.5 * np.eye(T.shape[0]) - D
    p_ref = oracle.lu_solve(A, b)
    inc_obs = np.exp(1j * k * obs[:, 2])
    w_ref = np.conj(inc_obs - oracle.eval_points(V, T, k, obs, x=p_ref)[0])
    r = np.linalg.norm(c[:, None, :] - obs[None, :, :], axis=2)
    pa_ref = oracle.lu_solve(A, ((np.exp(1j * k * r) / (4 * np.pi * r)) @ w_ref)[None, :])
    g = np.linspace(-2.0, 2.0, 7)
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    lat = lat[np.linalg.norm(lat, axis=1) > 1.2]
    # oracle composition
    inc = np.exp(1j * k * lat[:, 2])
    inc4 = np.stack([inc, 0 * inc, 0 * inc, 1j * k * inc], axis=1)
    p_f = inc - oracle.eval_points(V, T, k, lat, x=p_ref)[0]
    gp_f = inc4[:, 1:] - oracle.eval_points_grad(V, T, k, lat, x=p_ref)[0]
    d = lat[:, None, :] - obs[None, :, :]
    rr = np.linalg.norm(d, axis=2)
    e = np.exp(1j * k * rr) * w_ref[None, :]
    phi = np.sum(e / (4 * np.pi * rr), axis=1)
    gphi = np.einsum("pm,pmc->pc", e * (1j * k * rr - 1) / (4 * np.pi * rr ** 3), d)
    pa_f = phi - oracle.eval_points(V, T, k, lat, x=pa_ref)[0]
    gpa_f = gphi - oracle.eval_points_grad(V, T, k, lat, x=pa_ref)[0]
    T_ref = np.real(1.5 * np.sum(gp_f * gpa_f, axis=1) - k * k * p_f * pa_f)
    op = Operator(V, T, k, p=10, mode=mode, leaf_level=0 if mode == "direct64" else 3, max_nrhs=2)
    chain = op.state_and_adjoint(torch.from_numpy(b).cuda(), obs, inc_obs, tol=1e-10 if mode == "direct64" else 1e-8)
    Tg = op.topological_derivative(lat, chain, obs, inc4).cpu().numpy()
    assert rel(Tg, T_ref) <= tol
    op.close()
