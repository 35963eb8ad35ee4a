"""The coupled solve of Eq. (GMRES): (1/2 I - D + S C) x = b, vs the oracle's dense LU.

C stands in for the FEM block of Section 2.3 with a scalar membrane on the
scatterer's own surface mesh: P1 stiffness K and mass M on the vertices, the
factorised K - rho_s omega^2 M (step 1 of the paper's algorithm), N the
consistent load of the element pressures, and T the vertex-to-element average
scaled by rho_f omega^2.  The elastic FEM itself (tetrahedra, NETGEN meshes)
is not part of this library; the callback is where a caller's FEM plugs in.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1606_02383_gb300 import _lib, inputs
from paper_1606_02383_gb300.operator import Operator

pytestmark = pytest.mark.gpu

RHO_S_OMEGA2 = 2.0              # rho_s omega^2 of K - rho_s omega^2 M
KAPPA = 2.5                     # K = stiffness + KAPPA M keeps K - rho_s omega^2 M definite
BETA = 0.25 * (1.0 + 0.2j)      # rho_f omega^2 of the displacement-to-density map, with damping


def _membrane(V, T):
    """Dense (K - rho_s omega^2 M, N, T) of the P1 membrane on the mesh (FP64)."""
    nv, nt = V.shape[0], T.shape[0]
    K = np.zeros((nv, nv))
    M = np.zeros((nv, nv))
    Nl = np.zeros((nv, nt))
    Tm = np.zeros((nt, nv), dtype=np.complex128)
    for j, tri in enumerate(T):
        P = V[tri]
        A = 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
        E = np.array([P[2] - P[1], P[0] - P[2], P[1] - P[0]])  # edge opposite each vertex
        K[np.ix_(tri, tri)] += (E @ E.T) / (4.0 * A)
        M[np.ix_(tri, tri)] += A / 12.0 * (np.ones((3, 3)) + np.eye(3))
        Nl[tri, j] += A / 3.0
        Tm[j, tri] = BETA / 3.0
    return K + (KAPPA - RHO_S_OMEGA2) * M, Nl, Tm


def _rhs(V, T, k):
    c, _, _, _ = oracle.geometry(V, T)
    pw = inputs.plane_wave(c, k)
    r = np.linalg.norm(c - np.array([0.0, 0.0, 3.0]), axis=1)
    ps = np.exp(1j * k * r) / (4 * np.pi * r)
    return np.stack([pw, ps / np.linalg.norm(ps) * np.linalg.norm(pw)])


def _torch_coupling(Kw, Nl, Tm):
    """The callback: y = T (K - rho_s omega^2 M)^{-1} N x on the GPU, K - rho_s omega^2 M factorised once."""
    LU, piv = torch.linalg.lu_factor(torch.from_numpy(Kw.astype(np.complex128)).cuda())
    Nd = torch.from_numpy(Nl.astype(np.complex128)).cuda()
    Td = torch.from_numpy(Tm).cuda()
    calls = [0]

    def coupling(cx, cy):
        z = Nd @ cx.T                                 # step 2(a): nodal loads [nv, nrhs]
        u = torch.linalg.lu_solve(LU, piv, z)         # step 2(b): the factorised FEM solve
        cy.copy_((Td @ u).T)                          # normal-derivative density per element
        calls[0] += 1

    return coupling, calls


@pytest.mark.parametrize("mode,p,tol,tol_lu", [("direct64", 0, 1e-10, 1e-8), ("mixed", 10, 1e-7, 1e-5)])
def test_coupled_solve_vs_dense_lu(cuda_ok, mode, p, tol, tol_lu):
    V, T = inputs.icosphere(3)
    k = 1.0
    b = _rhs(V, T, k)
    S, D = oracle.assemble(V, T, k)
    Kw, Nl, Tm = _membrane(V, T)
    C = Tm @ np.linalg.solve(Kw, Nl)
    A = 0.5 * np.eye(T.shape[0]) - D
    ref = oracle.lu_solve(A + S @ C, b)
    ref0 = oracle.lu_solve(A, b)
    # the coupling term changes the answer: the test is not the rigid case in disguise
    assert np.linalg.norm(ref - ref0) / np.linalg.norm(ref) > 0.05

    op = Operator(V, T, k, p=p, mode=mode, leaf_level=3 if mode == "mixed" else 0)
    coupling, calls = _torch_coupling(Kw, Nl, Tm)
    x, iters, relres = op.solve(torch.from_numpy(b).cuda(), tol=tol, max_iter=200, restart=50, coupling=coupling)
    x = x.cpu().numpy()
    assert np.all(relres <= tol)
    assert calls[0] >= iters      # one map per matrix-vector product
    for q in range(b.shape[0]):
        assert np.linalg.norm(x[q] - ref[q]) / np.linalg.norm(ref[q]) <= tol_lu


def test_coupled_zero_map_is_the_plain_solve(cuda_ok):
    """C = 0 gives the rigid system: the same iterates as the plain host-driven solve."""
    V, T = inputs.icosphere(3)
    k = 1.0
    b = torch.from_numpy(_rhs(V, T, k)).cuda()
    op = Operator(V, T, k, mode="direct64")
    x0, i0, r0 = op.solve(b, tol=1e-10, max_iter=100, restart=100, driver="host")
    x1, i1, r1 = op.solve(b, tol=1e-10, max_iter=100, restart=100, coupling=lambda cx, cy: cy.zero_())
    assert i0 == i1
    assert torch.linalg.norm(x1 - x0) / torch.linalg.norm(x0) <= 1e-12


def test_coupled_callback_errors(cuda_ok):
    V, T = inputs.icosphere(2)
    op = Operator(V, T, 1.0, mode="direct64")
    b = torch.ones((1, T.shape[0]), dtype=torch.complex128, device="cuda")

    def bad(cx, cy):
        raise ValueError("coupling failed")

    with pytest.raises(ValueError, match="coupling failed"):
        op.solve(b, tol=1e-8, coupling=bad)
    with pytest.raises(_lib.BemError) as e:
        op.solve(b, tol=1e-8, coupling=lambda cx, cy: cy.zero_(), driver="graph_only")
    assert e.value.code == _lib.BEM_ERR_UNSUPPORTED
    # the handle stays usable after both failures
    x, iters, rel = op.solve(b, tol=1e-8)
    assert rel[0] <= 1e-8
