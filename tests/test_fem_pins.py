"""Pins of the elastic FEM oracle (oracle/fem.py, Section 2.3's body half)
against what P1 elements and the geometry fix exactly:

- the Kuhn split: six positive tetrahedra per voxel whose volumes add up to
  the voxels', a closed boundary (every edge in two triangles, opposite
  directions) with outward normals (sum n A = 0, and sum (c.n) A / 3 is the
  volume by the divergence theorem);
- K annihilates the six rigid motions;
- the patch test: a linear displacement is exact for P1, so K u equals the
  boundary load of its constant stress: for u = -p0 x / (3 lambda + 2 mu)
  (uniform compression) that is -N p0, and for a pure shear the load of
  sigma n on every triangle;
- M integrates products of P1 fields exactly: u.M u = int |u|^2 for a
  translation (the volume) and for u = x (sums of x^2 over the voxels);
- the coupling map C = rho_f omega^2 Avg (K - rho_s omega^2 M)^{-1} (-N)
  applied to a vector equals its dense matrix, and a mistake planted in the
  oracle (the mass factor, the load sign) fails one of the checks above.
"""
import numpy as np
import pytest

from oracle import fem


def _sphere_mask(n, r):
    g = np.arange(n) - (n - 1) / 2.0
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    return X ** 2 + Y ** 2 + Z ** 2 <= r * r


@pytest.mark.parametrize("mask", [np.ones((1, 1, 1), bool), np.ones((3, 2, 2), bool), _sphere_mask(8, 3.6)])
def test_voxel_mesh_is_closed_and_outward(mask):
    h = 0.25
    nodes, tets, tris = fem.voxel_tets(mask, h=h, origin=(-1.0, 0.5, 2.0))
    assert tets.shape[0] == 6 * int(mask.sum())
    vols = [fem.shape_gradients(nodes[t])[0] for t in tets]
    assert min(vols) > 0
    assert abs(sum(vols) - mask.sum() * h ** 3) <= 1e-12
    # every directed edge appears once, its reverse once
    edges = {}
    for t in tris:
        for a in range(3):
            e = (int(t[a]), int(t[(a + 1) % 3]))
            edges[e] = edges.get(e, 0) + 1
    assert all(c == 1 for c in edges.values())
    assert all((b, a) in edges for (a, b) in edges)
    P = nodes[tris]
    cr = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    assert np.abs(cr.sum(axis=0)).max() <= 1e-12
    vol = np.einsum("ij,ij->", P.mean(axis=1), cr) / 6.0
    assert abs(vol - mask.sum() * h ** 3) <= 1e-12


def _body(mask=None, h=0.3):
    mask = _sphere_mask(7, 3.1) if mask is None else mask
    return fem.voxel_tets(mask, h=h, origin=(0.2, -0.4, 0.1))


def test_stiffness_annihilates_rigid_motions():
    nodes, tets, _ = _body()
    K, _ = fem.assemble(nodes, tets, 2.0, 0.7)
    scale = abs(K).max() * np.abs(nodes).max()
    for i in range(3):
        u = np.zeros_like(nodes)
        u[:, i] = 1.0
        assert np.abs(K @ u.ravel()).max() <= 1e-12 * scale
        w = np.zeros(3)
        w[i] = 1.0
        assert np.abs(K @ np.cross(w, nodes).ravel()).max() <= 1e-12 * scale


def _traction_load(nodes, tris, sigma):
    f = np.zeros_like(nodes)
    P = nodes[tris]
    cr = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])  # 2 A n
    for j, t in enumerate(tris):
        f[t] += (sigma @ cr[j]) / 6.0
    return f.ravel()


def test_patch_test_uniform_compression_and_shear():
    lam, mu, p0 = 2.0, 0.7, 1.3
    nodes, tets, tris = _body()
    K, _ = fem.assemble(nodes, tets, lam, mu)
    N, _ = fem.surface_maps(nodes, tris)
    # uniform pressure p0 on the body: u = -p0 x / (3 lambda + 2 mu), load -N p0
    u = -p0 * nodes / (3 * lam + 2 * mu)
    load = -(N @ np.full(tris.shape[0], p0))
    assert np.abs(K @ u.ravel() - load).max() <= 1e-12 * np.abs(load).max()
    # pure shear e_01 = s: sigma = 2 mu e
    s = 0.4
    E = np.zeros((3, 3))
    E[0, 1] = E[1, 0] = s
    u = nodes @ E.T
    f = _traction_load(nodes, tris, 2 * mu * E)
    assert np.abs(K @ u.ravel() - f).max() <= 1e-12 * np.abs(f).max()


def test_mass_integrates_p1_products():
    h = 0.3
    mask = _sphere_mask(7, 3.1)
    nodes, tets, _ = _body(mask, h)
    _, M = fem.assemble(nodes, tets, 1.0, 1.0)
    vol = mask.sum() * h ** 3
    u = np.zeros_like(nodes)
    u[:, 2] = 1.0
    assert abs(u.ravel() @ (M @ u.ravel()) - vol) <= 1e-12 * vol
    # u = (x, 0, 0): int x^2 over every voxel [a, a + h] = ((a + h)^3 - a^3) h^2 / 3
    u = np.zeros_like(nodes)
    u[:, 0] = nodes[:, 0]
    a = 0.2 + h * np.argwhere(mask)[:, 0]
    exact = np.sum(((a + h) ** 3 - a ** 3) / 3.0) * h * h
    assert abs(u.ravel() @ (M @ u.ravel()) - exact) <= 1e-12 * exact


def test_coupling_map_matches_its_matrix():
    nodes, tets, tris = _body(_sphere_mask(5, 2.2), 0.4)
    body = fem.Body(nodes, tets, tris, lam=2.0, mu=0.7, rho_s=1.5, rho_f=0.8, omega=0.9)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(tris.shape[0]) + 1j * rng.standard_normal(tris.shape[0])
    C = body.matrix()
    assert np.abs(body.couple(x) - C @ x).max() <= 1e-12 * np.abs(C @ x).max()
    # the solve inverts K - rho_s omega^2 M
    b = rng.standard_normal(3 * nodes.shape[0])
    assert np.abs(body.A @ body.solve(b) - b).max() <= 1e-10 * np.abs(b).max()


def test_planted_mistakes_fail_the_pins(monkeypatch):
    """The pins catch a wrong mass factor and a wrong load sign."""
    lam, mu, p0 = 2.0, 0.7, 1.3
    nodes, tets, tris = _body()
    orig = fem.element_matrices

    def wrong_mass(X, lam_, mu_):
        Ke, Me = orig(X, lam_, mu_)
        return Ke, Me * (24.0 / 20.0)

    monkeypatch.setattr(fem, "element_matrices", wrong_mass)
    _, M = fem.assemble(nodes, tets, lam, mu)
    u = np.zeros_like(nodes)
    u[:, 2] = 1.0
    vol = sum(fem.shape_gradients(nodes[t])[0] for t in tets)
    assert abs(u.ravel() @ (M @ u.ravel()) - vol) > 1e-3 * vol
    monkeypatch.setattr(fem, "element_matrices", orig)
    K, _ = fem.assemble(nodes, tets, lam, mu)
    N, _ = fem.surface_maps(nodes, tris)
    u = -p0 * nodes / (3 * lam + 2 * mu)
    wrong_load = N @ np.full(tris.shape[0], p0)  # the other sign
    assert np.abs(K @ u.ravel() - wrong_load).max() > 0.5 * np.abs(wrong_load).max()


@pytest.mark.parametrize("mask", [np.ones((2, 3, 1), bool), _sphere_mask(7, 3.1)])
def test_shared_voxel_generator_matches_the_oracle_mesher(mask):
    """inputs.voxel_body (the seeded generator both sides take their bodies
    from) gives the oracle mesher's nodes, tetrahedra and boundary faces (up to
    order), and its jittered nodes keep every tetrahedron positive."""
    from paper_1606_02383_gb300 import inputs
    a = inputs.voxel_body(mask, 0.3, (0.1, -0.2, 0.4))
    b = fem.voxel_tets(mask, 0.3, (0.1, -0.2, 0.4))
    assert np.array_equal(a[0], b[0])
    assert sorted(map(tuple, np.sort(a[1], axis=1))) == sorted(map(tuple, np.sort(b[1], axis=1)))
    # faces equal as oriented triangles: the same cyclic order
    def canon(t):
        k = int(np.argmin(t))
        return tuple(int(v) for v in np.roll(t, -k))
    assert sorted(canon(t) for t in a[2]) == sorted(canon(t) for t in b[2])
    nodes, tets, _ = inputs.voxel_body(mask, 0.3, jitter=0.05, seed=1)
    assert min(fem.shape_gradients(nodes[t])[0] for t in tets) > 0
