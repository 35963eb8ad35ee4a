"""Pins of the coupled acoustic-elastic problem (Section 2.1, solved by
Section 2.3's BEM-FEM system) against the exact solution for an elastic
sphere, so that the oracle's reading of the coupling (the load -N p of the
traction t = -p n, the element mean of u.n that the single layer takes, the
composition (1/2 I - D + S C) p = p_src) is fixed by the physics rather than
by the oracle itself.

- The sphere's series solution (oracle/closed_forms.py, one 3 x 3 system of
  the boundary conditions per order) is pinned on its own: the lossless
  sphere's S-matrix entries 1 + 2 t_n have modulus 1; a very stiff and heavy
  sphere gives the rigid (sound-hard) sphere's coefficients; mu -> 0 gives the
  fluid sphere of bulk modulus lambda, a separate closed form, at O(mu).
- The oracle's coupled solve (dense S, D, the FEM oracle's C, LU) on
  tetrahedral balls whose boundaries are icospheres converges to the series
  solution's surface pressure (1.4% at 320 triangles, 0.51% at 1,280), where
  the elastic term moves the answer by 18% from the rigid sphere's; the other
  sign of the load gives 46%.
"""
import numpy as np
import pytest
from scipy import special as sp

import oracle
from oracle import closed_forms as cf
from oracle import fem
from paper_1606_02383_gb300 import inputs

LAM, MU, RHO_S, RHO_F, C_F, OMEGA, A = 2.0, 1.0, 2.0, 1.0, 1.0, 2.0, 0.5


def test_elastic_sphere_series_pins():
    k = OMEGA / C_F
    for n in range(8):
        An, _, _ = cf.elastic_sphere_coefficients(n, OMEGA, A, LAM, MU, RHO_S, RHO_F, C_F)
        t = An / ((2 * n + 1) * 1j ** n)
        assert abs(abs(1 + 2 * t) - 1.0) <= 1e-12
        # rigid limit: stiffness and density scaled up together (wave speeds kept)
        Ar, _, _ = cf.elastic_sphere_coefficients(n, OMEGA, A, LAM * 1e8, MU * 1e8, RHO_S * 1e8, RHO_F, C_F)
        rigid = -(2 * n + 1) * (1j ** n) * sp.spherical_jn(n, k * A, True) / (
            sp.spherical_jn(n, k * A, True) + 1j * sp.spherical_yn(n, k * A, True))
        assert abs(Ar - rigid) <= 1e-7 * abs(rigid)
        # fluid limit: the error of the mu -> 0 sphere against the fluid sphere falls like mu
        Af = cf.fluid_sphere_coefficient(n, OMEGA, A, LAM, RHO_S, RHO_F, C_F)
        e4 = abs(cf.elastic_sphere_coefficients(n, OMEGA, A, LAM, MU * 1e-4, RHO_S, RHO_F, C_F)[0] - Af)
        e6 = abs(cf.elastic_sphere_coefficients(n, OMEGA, A, LAM, MU * 1e-6, RHO_S, RHO_F, C_F)[0] - Af)
        # (floors of 1e-12: the high orders' coefficients are below 1e-10)
        assert e6 <= 2e-2 * e4 + 1e-12 and e6 <= 1e-4 * abs(Af) + 1e-12


def test_ball_tetrahedra_are_conforming():
    nodes, tets, tris = inputs.ball_tets(2, A, 3)
    assert min(fem.shape_gradients(nodes[t])[0] for t in tets) > 0
    faces = {}
    for t in tets:
        for skip in range(4):
            key = tuple(sorted(int(t[a]) for a in range(4) if a != skip))
            faces[key] = faces.get(key, 0) + 1
    assert max(faces.values()) == 2
    assert {f for f, c in faces.items() if c == 1} == {tuple(sorted(int(v) for v in t)) for t in tris}
    P = nodes[tris]
    out = np.einsum("ij,ij->i", np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), P.mean(axis=1))
    assert np.all(out > 0)


def _coupled_error(level, layers, sign=1.0):
    nodes, tets, tris = inputs.ball_tets(level, A, layers)
    k = OMEGA / C_F
    c = inputs.centroids(nodes, tris)
    b = np.exp(1j * k * c[:, 2])[None]
    S, D = oracle.assemble(nodes, tris, k)
    C = sign * fem.Body(nodes, tets, tris, LAM, MU, RHO_S, RHO_F, OMEGA).matrix()
    p = oracle.lu_solve(0.5 * np.eye(tris.shape[0]) - D + S @ C, b)[0]
    ref = cf.elastic_sphere_surface(OMEGA, A, LAM, MU, RHO_S, RHO_F, C_F, c[:, 2] / np.linalg.norm(c, axis=1))
    return float(np.linalg.norm(p - ref) / np.linalg.norm(ref))


def test_oracle_coupled_solve_converges_to_the_elastic_sphere():
    e2 = _coupled_error(2, 3)
    e3 = _coupled_error(3, 5)
    assert e2 <= 0.03 and e3 <= 0.01, (e2, e3)
    assert e3 <= 0.5 * e2, (e2, e3)
    # the load with the other sign is far off: the reading is fixed by the physics
    assert _coupled_error(2, 3, sign=-1.0) >= 0.3
