"""Marching-tetrahedra iso-surface of a grid function (test infrastructure only:
only the tests, the smoke check and the bench's CPU leg use it).

The boundary {phi = t} of the level-set region {phi > t} (Section 2.4: the
elastic body is where phi > 0 and its boundary is phi = 0), written out from
its definition in plain Python over the cut edges and the mixed cubes:

- grid point (i, j, k) sits at lo + (i, j, k) h and holds phi[i, j, k]; it is
  inside when phi > t;
- every cube splits into 6 tetrahedra, one per order (p0, p1, p2) of the axes
  in the order of PERMS, with corners 0, e_p0, e_p0 + e_p1 and (1, 1, 1);
- every edge of that split runs from a grid point g along one of the 7 steps
  in DIRS.  An edge with exactly one end inside holds one vertex, at
  a + s (b - a) from its lower end a, s = (t - phi_a) / (phi_b - phi_a)
  clamped to [0.02, 0.98];
- a tetrahedron with one corner alone on its side (1 or 3 corners inside)
  gives the triangle of the cuts of the three edges at that corner, in
  corner order; with corners a < b inside and c < d outside it gives the
  quadrilateral cut(a,c), cut(a,d), cut(b,d), cut(b,c), split along its
  first diagonal into (q0, q1, q2) and (q0, q2, q3);
- a triangle whose normal (B - A) x (C - A) points against
  mean(outside corners) - mean(inside corners) (taken times nin (4 - nin),
  an integer vector with the same direction) has its last two vertices
  swapped, so every triangle faces out of {phi > t}.

Output order: vertices by (g, step), triangles by (cube, tetrahedron, piece),
with g and the cube numbered i-major.
"""
from __future__ import annotations

import numpy as np

DIRS = ((1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1))
PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def _corners(p):
    out, v = [(0, 0, 0)], [0, 0, 0]
    for axis in PERMS[p]:
        v = list(v)
        v[axis] = 1
        out.append(tuple(v))
    return out


def isosurface(phi, lo, h, t):
    """(vertices [nv, 3] float64, triangles [nt, 3] int64) of {phi = t}."""
    phi = np.asarray(phi, dtype=np.float64)
    n0, n1, n2 = phi.shape
    lo = [float(x) for x in lo]
    h, t = float(h), float(t)
    inside = phi > t

    # vertices, one per cut edge, in (g, step) order
    cut = []
    for d, (a, b, c) in enumerate(DIRS):
        lower = inside[:n0 - a, :n1 - b, :n2 - c]
        upper = inside[a:, b:, c:]
        for i, j, k in zip(*np.nonzero(lower != upper)):
            i, j, k = int(i), int(j), int(k)
            cut.append(((i * n1 + j) * n2 + k, d, i, j, k))
    cut.sort()
    vid, verts = {}, []
    for g, d, i, j, k in cut:
        a, b, c = DIRS[d]
        fa, fb = float(phi[i, j, k]), float(phi[i + a, j + b, k + c])
        s = (t - fa) / (fb - fa)
        s = min(max(s, 0.02), 0.98)
        pa = (lo[0] + i * h, lo[1] + j * h, lo[2] + k * h)
        pb = (lo[0] + (i + a) * h, lo[1] + (j + b) * h, lo[2] + (k + c) * h)
        verts.append(tuple(pa[x] + s * (pb[x] - pa[x]) for x in range(3)))
        vid[(g, d)] = len(verts) - 1

    # triangles of the mixed cubes, in (cube, tetrahedron, piece) order
    corners = [_corners(p) for p in range(6)]
    c8 = [inside[a:n0 - 1 + a, b:n1 - 1 + b, c:n2 - 1 + c] for a in (0, 1) for b in (0, 1) for c in (0, 1)]
    mixed = np.logical_or.reduce(c8) & ~np.logical_and.reduce(c8)
    tris = []
    for i, j, k in zip(*np.nonzero(mixed)):
        i, j, k = int(i), int(j), int(k)
        for p in range(6):
            cs = corners[p]
            ins = [q for q in range(4) if inside[i + cs[q][0], j + cs[q][1], k + cs[q][2]]]
            outs = [q for q in range(4) if q not in ins]
            if len(ins) in (0, 4):
                continue

            def edge(q, r):
                u, w = (cs[q], cs[r]) if q < r else (cs[r], cs[q])
                g = ((i + u[0]) * n1 + (j + u[1])) * n2 + (k + u[2])
                return vid[(g, DIRS.index((w[0] - u[0], w[1] - u[1], w[2] - u[2])))]

            if len(ins) in (1, 3):
                lone, rest = (ins[0], outs) if len(ins) == 1 else (outs[0], ins)
                pieces = [[edge(lone, r) for r in rest]]
            else:
                a, b = ins
                c, d = outs
                q = [edge(a, c), edge(a, d), edge(b, d), edge(b, c)]
                pieces = [[q[0], q[1], q[2]], [q[0], q[2], q[3]]]
            # nin (4 - nin) (mean(outside corners) - mean(inside corners)): the
            # positive factor leaves the sign of the test alone
            away = [float(len(ins) * sum(cs[q][x] for q in outs) - len(outs) * sum(cs[q][x] for q in ins))
                    for x in range(3)]
            for tri in pieces:
                A, B, C = (verts[v] for v in tri)
                e1 = [B[x] - A[x] for x in range(3)]
                e2 = [C[x] - A[x] for x in range(3)]
                nrm = [e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]]
                if nrm[0] * away[0] + nrm[1] * away[1] + nrm[2] * away[2] < 0.0:
                    tri = [tri[0], tri[2], tri[1]]
                tris.append(tri)
    V = np.asarray(verts, dtype=np.float64).reshape(-1, 3)
    T = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
    return V, T
