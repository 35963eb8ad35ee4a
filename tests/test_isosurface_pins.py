"""Pins of the oracle's marching-tetrahedra iso-surface (no GPU): exact sections
of a linear function, closed surfaces with the Euler characteristic of their
topology, enclosed volume and area against the exact shapes, and agreement
with the workload's own host mesher."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
from paper_1606_02383_gb300 import inputs


def _grid(n, lo, hi):
    x = np.linspace(lo, hi, n)
    return np.meshgrid(x, x, x, indexing="ij"), np.array([lo, lo, lo]), x[1] - x[0]


def _areas(V, T):
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    return 0.5 * np.cross(b - a, c - a)


def _volume(V, T):
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    return np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0


def _closed_oriented(T):
    """Every edge in exactly two triangles, once in each direction; returns V - E + F."""
    directed = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]])
    assert len({tuple(e) for e in directed.tolist()}) == len(directed), "a directed edge repeats"
    undirected = {tuple(sorted(e)) for e in directed.tolist()}
    assert 2 * len(undirected) == len(directed), "an edge is not shared by exactly two triangles"
    nv = len(np.unique(T))
    return nv - len(undirected) + len(T)


def test_plane_section_is_exact():
    """phi = z: every cut sits at s = 1/2 of its edge, the section is the plane z = t
    over the whole box (area 4) and faces -z (out of z > t)."""
    (X, Y, Z), lo, h = _grid(9, -1.0, 1.0)
    V, T = oracle.isosurface(Z, lo, h, 0.125)
    assert np.all(V[:, 2] == 0.125)
    A = _areas(V, T)
    assert abs(np.linalg.norm(A, axis=1).sum() - 4.0) < 1e-13
    assert np.all(A[:, 2] < 0) and np.abs(A[:, :2]).max() < 1e-15
    # one layer of 8 x 8 cubes is cut; in each, the two tetrahedra that step along z
    # first or last have 3 or 1 corners above the plane (one triangle each) and the
    # two that step along z second have 2 (two triangles each): 8 per cube
    assert len(T) == 8 * 8 * 8


def test_sphere_is_closed_with_its_volume_and_area():
    (X, Y, Z), lo, h = _grid(41, -1.5, 1.5)
    V, T = oracle.isosurface(1.0 - (X * X + Y * Y + Z * Z), lo, h, 0.0)
    assert _closed_oriented(T) == 2
    vol = _volume(V, T)  # positive: the triangles face outwards
    assert abs(vol - 4.0 * np.pi / 3.0) / (4.0 * np.pi / 3.0) < 0.02
    area = np.linalg.norm(_areas(V, T), axis=1).sum()
    assert abs(area - 4.0 * np.pi) / (4.0 * np.pi) < 0.02


def test_torus_and_two_spheres_topology():
    (X, Y, Z), lo, h = _grid(49, -1.6, 1.6)
    torus = 0.4 ** 2 - (np.sqrt(X * X + Y * Y) - 1.0) ** 2 - Z * Z
    V, T = oracle.isosurface(torus, lo, h, 0.0)
    assert _closed_oriented(T) == 0
    assert abs(_volume(V, T) - 2 * np.pi ** 2 * 1.0 * 0.4 ** 2) / (2 * np.pi ** 2 * 0.16) < 0.03
    two = np.maximum(0.5 ** 2 - ((X - 0.8) ** 2 + Y * Y + Z * Z), 0.5 ** 2 - ((X + 0.8) ** 2 + Y * Y + Z * Z))
    V, T = oracle.isosurface(two, lo, h, 0.0)
    assert _closed_oriented(T) == 4


def test_single_corner_cube_and_empty_levels():
    phi = np.zeros((2, 2, 2))
    phi[0, 0, 0] = 1.0
    V, T = oracle.isosurface(phi, (0.0, 0.0, 0.0), 1.0, 0.5)
    # every edge from the corner is cut (7 vertices, all at s = 1/2); each of the 6
    # tetrahedra holds the corner alone: a fan of 6 triangles around the diagonal
    assert V.shape == (7, 3) and T.shape == (6, 3)
    assert np.allclose(V, 0.5 * np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [1, 0, 1], [0, 1, 1], [1, 1, 1]]))
    assert np.all(np.einsum("ij,j->i", _areas(V, T), [1.0, 1.0, 1.0]) > 0)  # away from the corner
    for t in (2.0, -1.0):  # nothing inside / everything inside
        V, T = oracle.isosurface(phi, (0.0, 0.0, 0.0), 1.0, t)
        assert V.shape == (0, 3) and T.shape == (0, 3)


def test_clamp_keeps_cut_points_off_the_grid_points():
    phi = np.zeros((2, 2, 2))
    phi[0, 0, 0] = 1.0
    V, _ = oracle.isosurface(phi, (0.0, 0.0, 0.0), 1.0, 1.0 - 1e-9)  # s would be 1e-9
    assert np.allclose(np.linalg.norm(V, axis=1) / np.linalg.norm(
        np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [1, 0, 1], [0, 1, 1], [1, 1, 1]]), axis=1), 0.02)


@pytest.mark.parametrize("grid", [24, 64])
def test_agrees_with_the_workload_mesher(grid):
    """The workload's host mesher is a second implementation of the same surface
    (it interpolates from whichever end it meets first, so only rounding differs)."""
    phi, lo, h = inputs.level_set_function(0, 20, grid)
    t = float(np.median(phi)) if grid < 64 else inputs.level_set_level()
    V, T = oracle.isosurface(phi, lo, h, t)
    V2, T2 = inputs._marching_tets(phi, lo, h, t)
    assert V.shape == V2.shape and T.shape == T2.shape
    assert np.abs(np.sort(V, axis=0) - np.sort(V2, axis=0)).max() < 1e-14
    assert abs(_volume(V, T) - _volume(V2, T2)) < 1e-12
    # the same oriented triangles: map the mesher's vertices onto the oracle's
    dist, idx = cKDTree(V).query(V2)
    assert dist.max() < 1e-14 and len(set(idx.tolist())) == len(V)
    assert _oriented_set(T) == _oriented_set(idx[T2])


def _oriented_set(T):
    """Triangles rotated so their smallest index comes first (orientation kept)."""
    out = set()
    for a, b, c in np.asarray(T).tolist():
        m = min(a, b, c)
        out.add((a, b, c) if m == a else ((b, c, a) if m == b else (c, a, b)))
    return out
