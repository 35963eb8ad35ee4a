"""Adjoint double layer D' and hypersingular operator H on flat triangles with
centroid collocation (test infrastructure only: only the tests, the smoke
check and the bench's CPU leg use it).

With G = exp(ikr)/(4 pi r), d = y - x, r = |d|,
F = exp(ikr)(ikr - 1)/(4 pi r^3) and Hs = exp(ikr)(3 - 3ikr - k^2 r^2)/(4 pi r^5):

    dG/dn_x          = -F (d . n_x)
    d^2 G/dn_x dn_y  = -Hs (d . n_x)(d . n_y) - F (n_x . n_y)

    D'_ij = int_{Gamma_j} dG(x_i - y)/dn_x,   H_ij = int_{Gamma_j} d^2 G(x_i - y)/dn_x dn_y.

They complete the Burton-Miller form of the sound-hard problem: with the
normals pointing into the fluid, the total pressure p on Gamma satisfies
(1/2 I - D) p = p_inc (the equation the library solves; Section 2.3 with the
FEM term absent) and H p = -dp_inc/dn (the normal derivative of the same
representation, which has no jump).  Their combination

    (1/2 I - D + alpha H) p = p_inc - alpha dp_inc/dn,   alpha = i / k,

is uniquely solvable at the interior Dirichlet eigenvalues where the first
equation alone is singular (Section 1 of the paper notes those frequencies).

Rules (the paper gives none; the reading written out here):
- off the element, the 3-point rule of the library on the element split
  uniformly L times, with L = 4 within 2 h_j of the centroid c_j, 3 within
  4 h_j, 2 within 8 h_j and 0 beyond (h_j the longest edge): the 1/r^3
  kernel of H needs deeper splits than S and D;
- on the element (j = i, flat): D'_ii = 0, and H_ii is the Hadamard finite
  part of -F over the triangle about its centroid.  In polar coordinates
  about the centroid the radial integral is exact, because
  d/dr[-exp(ikr)/r] = exp(ikr)(1 - ikr)/r^2, so
      H_ii = (1/(4 pi)) [2 pi i k - int_0^{2 pi} exp(ik R(theta)) / R(theta) dtheta],
  R(theta) the distance to the boundary along the ray, integrated edge by
  edge with 64-point Gauss-Legendre in the angle.
"""
from __future__ import annotations

import numpy as np

LEVELS = ((2.0, 4), (4.0, 3), (8.0, 2))
_BARY = np.array([[2 / 3, 1 / 6, 1 / 6], [1 / 6, 2 / 3, 1 / 6], [1 / 6, 1 / 6, 2 / 3]])


def _geometry(V, T):
    V = np.asarray(V, dtype=np.float64)
    T = np.asarray(T, dtype=np.int64)
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    cr = np.cross(b - a, c - a)
    area = 0.5 * np.linalg.norm(cr, axis=1)
    n = cr / (2.0 * area[:, None])
    cen = (a + b + c) / 3.0
    h = np.max(np.stack([np.linalg.norm(b - a, axis=1), np.linalg.norm(c - b, axis=1),
                         np.linalg.norm(a - c, axis=1)]), axis=0)
    return a, b, c, cen, area, n, h


def _rule_all(a, b, c, L):
    """Points [nt, 3 4^L, 3] and weights [nt, 3 4^L] of the 3-point rule on the
    L-fold uniform split of every triangle."""
    tri = np.stack([a, b, c], axis=1)[:, None]                      # [nt, 1, 3, 3]
    for _ in range(L):
        p, q, r = tri[:, :, 0], tri[:, :, 1], tri[:, :, 2]
        pq, qr, rp = 0.5 * (p + q), 0.5 * (q + r), 0.5 * (r + p)
        tri = np.concatenate([np.stack(s_, axis=2) for s_ in ((p, pq, rp), (pq, q, qr), (rp, qr, r), (pq, qr, rp))],
                             axis=1)
    pts = np.einsum("qk,nmkd->nmqd", _BARY, tri).reshape(tri.shape[0], -1, 3)
    ar = 0.5 * np.linalg.norm(np.cross(tri[:, :, 1] - tri[:, :, 0], tri[:, :, 2] - tri[:, :, 0]), axis=-1)
    return pts, np.repeat(ar / 3.0, 3, axis=1)


def _self_hypersingular(a, b, c, cen, k, nodes=64):
    t, w = np.polynomial.legendre.leggauss(nodes)
    total = 2.0 * np.pi * 1j * k
    for p, q in ((a, b), (b, c), (c, a)):
        e = q - p
        te = e / np.linalg.norm(e)
        foot = p + ((cen - p) @ te) * te
        u = foot - cen
        dist = np.linalg.norm(u)
        phi_a = np.arctan2((p - cen) @ te, dist)
        phi_b = np.arctan2((q - cen) @ te, dist)
        phi = 0.5 * (phi_b - phi_a) * t + 0.5 * (phi_b + phi_a)
        R = dist / np.cos(phi)
        total -= 0.5 * (phi_b - phi_a) * np.sum(w * np.exp(1j * k * R) / R)
    return total / (4.0 * np.pi)


def assemble(V, T, k):
    """Dense (D', H), complex [nt, nt]."""
    a, b, c, cen, area, n, h = _geometry(V, T)
    nt = len(area)
    Dp = np.zeros((nt, nt), dtype=np.complex128)
    H = np.zeros((nt, nt), dtype=np.complex128)
    # regular rule for every pair first (vectorised by rows), then the refined pairs
    P0 = np.einsum("qk,mkd->mqd", _BARY, np.stack([a, b, c], axis=1))        # [nt, 3, 3]
    w0 = np.repeat((area / 3.0)[:, None], 3, axis=1)                           # [nt, 3]
    for i0 in range(0, nt, 64):
        i1 = min(nt, i0 + 64)
        d = P0[None, :, :, :] - cen[i0:i1, None, None, :]                     # [bi, nt, 3, 3]
        r = np.linalg.norm(d, axis=-1)
        e = np.exp(1j * k * r)
        F = e * (1j * k * r - 1.0) / (4.0 * np.pi * r ** 3)
        Hs = e * (3.0 - 3.0j * k * r - (k * r) ** 2) / (4.0 * np.pi * r ** 5)
        dnx = np.einsum("ijqd,id->ijq", d, n[i0:i1])
        dny = np.einsum("ijqd,jd->ijq", d, n)
        nn = n[i0:i1] @ n.T                                                     # [bi, nt]
        Dp[i0:i1] = np.sum(w0[None] * (-F * dnx), axis=2)
        H[i0:i1] = np.sum(w0[None] * (-Hs * dnx * dny - F * nn[:, :, None]), axis=2)
    dist = np.linalg.norm(cen[:, None, :] - cen[None, :, :], axis=2)
    lev = np.zeros((nt, nt), dtype=np.int64)
    for f, L in reversed(LEVELS):
        lev[dist < f * h[None, :]] = L
    np.fill_diagonal(lev, 0)
    for L in sorted({L for _, L in LEVELS}):
        pts, w = _rule_all(a, b, c, L)
        for i in range(nt):
            js = np.nonzero(lev[i] == L)[0]
            if len(js) == 0:
                continue
            d = pts[js] - cen[i]                                                  # [m, P, 3]
            r = np.linalg.norm(d, axis=-1)
            e = np.exp(1j * k * r)
            F = e * (1j * k * r - 1.0) / (4.0 * np.pi * r ** 3)
            Hs = e * (3.0 - 3.0j * k * r - (k * r) ** 2) / (4.0 * np.pi * r ** 5)
            dnx = d @ n[i]
            dny = np.einsum("mpd,md->mp", d, n[js])
            Dp[i, js] = np.sum(w[js] * (-F * dnx), axis=1)
            H[i, js] = np.sum(w[js] * (-Hs * dnx * dny - F * (n[js] @ n[i])[:, None]), axis=1)
    for i in range(nt):
        Dp[i, i] = 0.0
        H[i, i] = _self_hypersingular(a[i], b[i], c[i], cen[i], k)
    return Dp, H
