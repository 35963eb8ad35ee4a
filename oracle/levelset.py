"""One step of the level-set update of Section 2.4 (test infrastructure only:
only the tests, the smoke check and the bench's CPU leg use it).

The fictitious-time evolution (Section 2.4) is

    d phi / dt = -C T_Omega  + tau L^2 lap phi   where phi <= 0 (the fluid, Omega),
    d phi / dt =  C T_Omegac + tau L^2 lap phi   where phi > 0  (the body, Omega^c),
    phi = phi_bar (< 0) on the boundary of the design box D,

solved by FEM on the voxels of the lattice that carries phi (Section 2.5,
steps 1, 2 and 9).  The paper leaves the discretisation to its reference;
the reading written out here:

- Q1 (trilinear) elements on the voxels of a uniform lattice with spacing h;
  K = int grad N_a . grad N_b and M = int N_a N_b, assembled element by
  element, each element matrix by 2-point Gauss quadrature per axis (exact
  for Q1 products);
- one step of length dt, implicit in the diffusion and explicit in the
  topological-derivative term F (F = -C T_Omega where phi <= 0, C T_Omegac
  where phi > 0):  (M / dt + tau L^2 K) phi_new = M (phi / dt + F) on the
  interior nodes, phi_new = phi_bar on the boundary nodes;
- phi_new is then clamped to [-1, 1], the range in which Section 2.4 defines
  Omega, Gamma and Omega^c.

The interior system is symmetric positive definite; it is solved with
scipy's conjugate gradients to a relative residual of 1e-13 (a library
primitive).
"""
from __future__ import annotations

import numpy as np
from scipy import sparse
from scipy.sparse import linalg as spla

_G = (0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0))  # 2-point Gauss on [0, 1]


def _element_matrices(h):
    """(Ke, Me), 8 x 8, corner a = (a0, a1, a2) in {0,1}^3 numbered a0 * 4 + a1 * 2 + a2."""
    corners = [(a0, a1, a2) for a0 in (0, 1) for a1 in (0, 1) for a2 in (0, 1)]
    Ke = np.zeros((8, 8))
    Me = np.zeros((8, 8))
    for gx in _G:
        for gy in _G:
            for gz in _G:
                q = (gx, gy, gz)
                w = h ** 3 / 8.0  # each of the 8 Gauss points carries an eighth of the voxel
                val = np.empty(8)
                grad = np.empty((8, 3))
                for a, c in enumerate(corners):
                    f = [q[d] if c[d] else 1.0 - q[d] for d in range(3)]       # 1-D hat values
                    df = [1.0 / h if c[d] else -1.0 / h for d in range(3)]     # their derivatives
                    val[a] = f[0] * f[1] * f[2]
                    grad[a] = (df[0] * f[1] * f[2], f[0] * df[1] * f[2], f[0] * f[1] * df[2])
                Ke += w * grad @ grad.T
                Me += w * np.outer(val, val)
    return Ke, Me


def assemble(shape, h):
    """Q1 stiffness and mass (scipy CSR) on a lattice of `shape` nodes with spacing h."""
    n0, n1, n2 = shape
    Ke, Me = _element_matrices(h)
    I, J, K = np.meshgrid(np.arange(n0 - 1), np.arange(n1 - 1), np.arange(n2 - 1), indexing="ij")
    base = ((I * n1 + J) * n2 + K).ravel()
    offs = np.array([(a0 * n1 + a1) * n2 + a2 for a0 in (0, 1) for a1 in (0, 1) for a2 in (0, 1)])
    nodes = base[:, None] + offs[None, :]                               # [elements, 8]
    rows = np.repeat(nodes, 8, axis=1).ravel()
    cols = np.tile(nodes, (1, 8)).ravel()
    n = n0 * n1 * n2
    Kg = sparse.coo_matrix((np.tile(Ke.ravel(), len(base)), (rows, cols)), shape=(n, n)).tocsr()
    Mg = sparse.coo_matrix((np.tile(Me.ravel(), len(base)), (rows, cols)), shape=(n, n)).tocsr()
    return Kg, Mg


def boundary_mask(shape):
    m = np.zeros(shape, dtype=bool)
    m[0, :, :] = m[-1, :, :] = m[:, 0, :] = m[:, -1, :] = m[:, :, 0] = m[:, :, -1] = True
    return m


def step(phi, T_omega, T_omegac, h, dt, C, tau, L, phi_bar):
    """phi after one step of the update; every array is the lattice's shape."""
    phi = np.asarray(phi, dtype=np.float64)
    shape = phi.shape
    Kg, Mg = assemble(shape, h)
    F = np.where(phi <= 0.0, -C * np.asarray(T_omega, dtype=np.float64), C * np.asarray(T_omegac, dtype=np.float64))
    A = (Mg / dt + (tau * L * L) * Kg).tocsr()
    rhs = Mg @ (phi.ravel() / dt + F.ravel())
    bnd = boundary_mask(shape).ravel()
    inner = ~bnd
    out = np.where(bnd, np.broadcast_to(np.asarray(phi_bar, dtype=np.float64), shape).ravel(), 0.0)
    # move the known boundary values to the right-hand side
    rhs_i = rhs[inner] - A[inner][:, bnd] @ out[bnd]
    A_ii = A[inner][:, inner]
    x0 = phi.ravel()[inner]
    x, info = spla.cg(A_ii, rhs_i, x0=x0, rtol=1e-13, atol=0.0, maxiter=10000)
    if info != 0:
        raise RuntimeError("conjugate gradients did not converge")
    out[inner] = x
    return np.clip(out, -1.0, 1.0).reshape(shape)
