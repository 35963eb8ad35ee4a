"""The FMM walk of the off-surface evaluation (bem_eval_points on FMM handles).

Each point walks the octree from level 2: boxes that do not touch the point's
box (and lie at least 4 h_max away from its finest-level box) go through their
multipoles, near leaves are summed element by element with the rules of the
direct sum.  Checked here:
  - adaptive trees (leaves on several levels: split per box and per region)
    against the oracle, value and gradient;
  - a 20,480-triangle sphere at ka = 5 on a lattice (inside and outside the
    sphere, inside and outside the root cube) against the same handle's
    direct sum, which the other evaluation tests pin to the oracle, and
    against the oracle on sampled points;
  - several right-hand sides at once (the far pass shares its radial and
    angular functions across them) against one at a time.
Tolerances: mixed mode 1e-5 (measured up to 3.2e-6 for gradients on the
adaptive trees), FP64 mode at order 16: 1e-7 (measured 6.7e-9).  On the
lattice, with orders from eps = 1e-5 and random densities, the FMM is held
to 5e-5 for values and 2e-4 for gradients: the orders are chosen for
collocation values, the field away from the surface has no singular near
part, so the same absolute truncation is a larger share of it (measured
1.8e-5 against the direct sum on a 64^3 lattice, 2.2e-5 on 100^3), and the
derivative of the order-n term carries a factor of about n / r, so the
gradient's truncation is several times the value's (measured 9.1e-5).  With
eps = 1e-7 both shrink with the orders.  For the smooth density of a solved
plane wave the lattice field is within 3e-6 of the direct sum.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1606_02383_gb300 import inputs
from paper_1606_02383_gb300.operator import Operator

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def two_spheres():
    V1, T1 = inputs.icosphere(3)
    V2, T2 = inputs.icosphere(3, 0.3, (1.3, 0.4, -0.2))
    return inputs.merge_meshes([(V1, T1), (V2, T2)])


@pytest.mark.parametrize("mode,leaf,tol", [("mixed", -2, 1e-5), ("mixed", -1, 1e-5), ("fp64", -2, 1e-7),
                                           ("fp64", -1, 1e-7)])
def test_walk_on_adaptive_trees(cuda_ok, mode, leaf, tol):
    V, T = two_spheres()
    n, k = T.shape[0], 2.0
    x = inputs.random_density(n, 1, seed=3, stream=0)
    y = inputs.random_density(n, 1, seed=3, stream=1)
    rng = np.random.default_rng(1)
    c, _, _, _ = oracle.geometry(V, T)
    idx = rng.choice(n, 100, replace=False)
    pts = np.concatenate([rng.uniform(-2.0, 2.5, size=(400, 3)), c[idx] + 0.01 * rng.normal(size=(100, 3))])
    op = Operator(V, T, k, p=16, mode=mode, leaf_level=leaf, leaf_target=16, max_nrhs=1)
    levels = {l for l in range(11) if op.info(200 + l) > 0}
    assert len(levels) >= 2, levels
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    u = op.eval_points(pts, xd, yd).cpu().numpy()
    assert rel(u, oracle.eval_points(V, T, k, pts, x=x, y=y)) <= tol
    g = op.eval_points(pts, xd, yd, gradient=True).cpu().numpy()
    assert rel(g, oracle.eval_points_grad(V, T, k, pts, x=x, y=y)) <= tol
    op.close()


@pytest.mark.parametrize("eps,tol_u,tol_g", [(1e-5, 5e-5, 2e-4), (1e-7, 5e-6, 2e-5)])
def test_walk_on_a_lattice_around_a_large_sphere(cuda_ok, eps, tol_u, tol_g):
    V, T = inputs.icosphere(5)
    n, k = T.shape[0], 5.0
    x = inputs.random_density(n, 1, seed=2, stream=0)
    y = inputs.random_density(n, 1, seed=2, stream=1)
    g = np.linspace(-2.0, 2.0, 40)
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    lat = lat[np.abs(np.linalg.norm(lat, axis=1) - 1.0) > 0.05]
    op = Operator(V, T, k, p=0, eps=eps, mode="mixed", max_nrhs=1)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    u = op.eval_points(lat, xd, yd, value_and_gradient=True).cpu().numpy()[0]
    ud = op.eval_points(lat, xd, yd, value_and_gradient=True, direct=True).cpu().numpy()[0]
    eu, eg = rel(u[:, 0], ud[:, 0]), rel(u[:, 1:], ud[:, 1:])
    assert eu <= tol_u and eg <= tol_g, (eu, eg)
    smp = np.random.default_rng(0).choice(lat.shape[0], 100, replace=False)
    assert rel(u[smp, 0], oracle.eval_points(V, T, k, lat[smp], x=x, y=y)[0]) <= tol_u
    op.close()


def test_walk_with_several_right_hand_sides(cuda_ok):
    """nrhs = 7 runs the far and near passes in chunks of 4, 2 and 1."""
    V, T = inputs.icosphere(4)
    n, k = T.shape[0], 3.0
    x = inputs.random_density(n, 7, seed=5, stream=0)
    y = inputs.random_density(n, 7, seed=5, stream=1)
    rng = np.random.default_rng(2)
    pts = rng.uniform(-2.0, 2.0, size=(3000, 3))
    pts = pts[np.abs(np.linalg.norm(pts, axis=1) - 1.0) > 0.05]
    op = Operator(V, T, k, p=12, mode="mixed", max_nrhs=7)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    u = op.eval_points(pts, xd, yd, value_and_gradient=True).cpu().numpy()
    for r in range(7):
        ur = op.eval_points(pts, xd[r:r + 1], yd[r:r + 1], value_and_gradient=True).cpu().numpy()[0]
        assert rel(u[r], ur) <= 1e-6
    ref = oracle.eval_points(V, T, k, pts[:200], x=x[:2], y=y[:2])
    assert rel(u[:2, :200, 0], ref) <= 1e-5
    op.close()
