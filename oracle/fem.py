"""The elastic half of Section 2.3's coupled solver (test infrastructure only:
only the tests, the smoke check and the bench's CPU leg use it).

Section 2.3 discretises the body Omega^c into tetrahedra whose boundary faces
are the BEM triangles, with P1 (locally linear) displacements and Galerkin
test functions, which gives the stiffness K, the mass M and the load matrix N
of the pressure on Gamma; the second block row of the coupled system gives
u = (K - rho_s omega^2 M)^{-1} (load), and Eq. (GMRES) keeps only the BEM
unknowns.  Readings written out here:

- the body is a set of voxels of a uniform lattice, each split into the six
  tetrahedra around its main diagonal (Kuhn's split: the same in every voxel,
  so neighbouring voxels share their face triangles); the BEM mesh is the set
  of tetrahedron faces that belong to one tetrahedron only, ordered so that
  the normal points out of the body (the paper meshes with NETGEN, which is
  not available);
- K_e[(a,i),(b,k)] = V_e (lambda d_i phi_a d_k phi_b + mu d_k phi_a d_i phi_b
  + mu delta_ik grad phi_a . grad phi_b) from C_ijkl of the isotropic tensor,
  M_e[(a,i),(b,k)] = delta_ik V_e (1 + delta_ab) / 20 (the exact integrals of
  P1 products), degrees of freedom numbered 3 a + i;
- the traction is t = -p n on Gamma (n out of the body), so the load of the
  piecewise constant pressure is -N p with N[(a,i), j] = n_ji A_j / 3 for the
  three corners a of triangle j; the paper's weak form prints the pressure
  term with the other sign, which the boundary condition t_i + p n_i = 0 does
  not allow;
- the single layer of Eq. (GMRES) acts on the BEM's piecewise constant
  densities, so q = rho_f omega^2 u.n enters as its element mean,
  (u.n)_j = n_j . (u_a + u_b + u_c) / 3 (the mean of the linear field over the
  triangle);
- C = rho_f omega^2 Avg (K - rho_s omega^2 M)^{-1} (-N), so Eq. (GMRES) reads
  (1/2 I - D + S C) p = p_src.

Assembly is element by element in numpy; the solve is scipy's sparse LU (a
library primitive).
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy import sparse
from scipy.sparse import linalg as spla

# the six tetrahedra of the unit cube around its diagonal (0,0,0)-(1,1,1): one
# per order of the three axes, walking one unit step along each in turn
_KUHN = [p for p in itertools.permutations(range(3))]


def voxel_tets(mask, h=1.0, origin=(0.0, 0.0, 0.0)):
    """Tetrahedra of the voxels where mask is true.

    Returns (nodes [n, 3] float64, tets [m, 4] int32 with positive volume,
    tris [t, 3] int32, the boundary faces with outward normals).  Nodes are the
    lattice points of the body's voxels, numbered in lexicographic order."""
    mask = np.asarray(mask, dtype=bool)
    n0, n1, n2 = mask.shape
    corner = np.zeros((n0 + 1, n1 + 1, n2 + 1), dtype=bool)
    for d in itertools.product((0, 1), repeat=3):
        corner[d[0]:d[0] + n0, d[1]:d[1] + n1, d[2]:d[2] + n2] |= mask
    ids = -np.ones(corner.shape, dtype=np.int64)
    pts = np.argwhere(corner)
    ids[tuple(pts.T)] = np.arange(pts.shape[0])
    nodes = np.asarray(origin, dtype=np.float64) + h * pts.astype(np.float64)
    tets = []
    for v in np.argwhere(mask):
        for perm in _KUHN:
            c = v.copy()
            path = [ids[tuple(c)]]
            for axis in perm:
                c[axis] += 1
                path.append(ids[tuple(c)])
            tets.append(path)
    tets = np.asarray(tets, dtype=np.int64)
    # positive orientation
    P = nodes[tets]
    vol = np.einsum("ij,ij->i", np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), P[:, 3] - P[:, 0])
    flip = vol < 0
    tets[flip, 2], tets[flip, 3] = tets[flip, 3].copy(), tets[flip, 2].copy()
    # boundary faces: the faces that occur once, oriented away from their tetrahedron
    faces = {}
    for t in tets:
        for skip in range(4):
            f = [t[a] for a in range(4) if a != skip]
            key = tuple(sorted(f))
            if key in faces:
                faces[key] = None
            else:
                faces[key] = (f, t[skip])
    tris = []
    for key, val in faces.items():
        if val is None:
            continue
        f, opp = val
        a, b, c = nodes[f[0]], nodes[f[1]], nodes[f[2]]
        if np.dot(np.cross(b - a, c - a), a - nodes[opp]) < 0:
            f = [f[0], f[2], f[1]]
        tris.append(f)
    return nodes, tets.astype(np.int32), np.asarray(tris, dtype=np.int32)


def shape_gradients(X):
    """(V, G): volume and the constant gradients G[a] of the four P1 functions of
    the tetrahedron with corners X[0..3]."""
    J = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)  # columns: edges
    V = np.linalg.det(J) / 6.0
    Jinv = np.linalg.inv(J)  # rows: gradients of the barycentric coordinates 1..3
    G = np.empty((4, 3))
    G[1:] = Jinv
    G[0] = -Jinv.sum(axis=0)
    return V, G


def element_matrices(X, lam, mu):
    """(Ke, Me), 12 x 12, degrees of freedom 3 a + i (Me without rho_s)."""
    V, G = shape_gradients(X)
    Ke = np.zeros((12, 12))
    Me = np.zeros((12, 12))
    for a in range(4):
        for b in range(4):
            gg = G[a] @ G[b]
            for i in range(3):
                for k in range(3):
                    Ke[3 * a + i, 3 * b + k] = V * (lam * G[a, i] * G[b, k] + mu * G[a, k] * G[b, i]
                                                    + (mu * gg if i == k else 0.0))
                    if i == k:
                        Me[3 * a + i, 3 * b + k] = V * (2.0 if a == b else 1.0) / 20.0
    return Ke, Me


def assemble(nodes, tets, lam, mu):
    """Sparse (K, M) of the P1 elastic body, 3 n x 3 n."""
    n = nodes.shape[0]
    rows, cols, kv, mv = [], [], [], []
    for t in tets:
        Ke, Me = element_matrices(nodes[t], lam, mu)
        dof = np.array([3 * a + i for a in t for i in range(3)])
        rows.append(np.repeat(dof, 12))
        cols.append(np.tile(dof, 12))
        kv.append(Ke.ravel())
        mv.append(Me.ravel())
    rows, cols = np.concatenate(rows), np.concatenate(cols)
    K = sparse.csr_matrix((np.concatenate(kv), (rows, cols)), shape=(3 * n, 3 * n))
    M = sparse.csr_matrix((np.concatenate(mv), (rows, cols)), shape=(3 * n, 3 * n))
    return K, M


def surface_maps(nodes, tris):
    """(N, Avg): N[(a,i), j] = n_ji A_j / 3 (the load of a unit pressure on
    triangle j), Avg[j, (a,i)] = n_ji / 3 (the mean of u.n over triangle j)."""
    n, nt = nodes.shape[0], tris.shape[0]
    P = nodes[tris]
    cr = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    A = 0.5 * np.linalg.norm(cr, axis=1)
    nrm = cr / (2.0 * A[:, None])
    r, c, v = [], [], []
    for j in range(nt):
        for a in tris[j]:
            for i in range(3):
                r.append(3 * a + i)
                c.append(j)
                v.append(nrm[j, i] * A[j] / 3.0)
    N = sparse.csr_matrix((v, (r, c)), shape=(3 * n, nt))
    Avg = sparse.csr_matrix((np.asarray(v) / np.repeat(A, 9), (c, r)), shape=(nt, 3 * n))
    return N, Avg


class Body:
    """The elastic body of Section 2.3: K - rho_s omega^2 M factorised once (the
    paper's step 1), then C x = rho_f omega^2 Avg (K - rho_s omega^2 M)^{-1} (-N x)."""

    def __init__(self, nodes, tets, tris, lam, mu, rho_s, rho_f, omega):
        K, M = assemble(nodes, tets, lam, mu)
        self.A = (K - rho_s * omega ** 2 * M).tocsc()
        self.N, self.Avg = surface_maps(nodes, tris)
        self.beta = rho_f * omega ** 2
        self._lu = spla.splu(self.A)

    def solve(self, b):
        """(K - rho_s omega^2 M)^{-1} b, b real or complex [3 n] or [3 n, m]."""
        b = np.asarray(b)
        if np.iscomplexobj(b):
            return self._lu.solve(np.ascontiguousarray(b.real)) + 1j * self._lu.solve(np.ascontiguousarray(b.imag))
        return self._lu.solve(np.ascontiguousarray(b, dtype=np.float64))

    def couple(self, x):
        """C x for element densities x [nt] (complex)."""
        u = self.solve(-(self.N @ x))
        return self.beta * (self.Avg @ u)

    def matrix(self):
        """Dense C (nt x nt, real)."""
        U = self.solve(-self.N.toarray())
        return self.beta * (self.Avg @ U)
