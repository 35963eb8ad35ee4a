"""Pins of the oracle's adjoint double layer D' and hypersingular operator H
(no GPU), the operators of the Burton-Miller formulation.

- H applied to a constant density vanishes on a closed surface at k -> 0 (the
  double layer of a constant is piecewise constant, so its normal derivative
  is zero): this fixes the finite-part self term, which carries most of each row.
- The sphere eigenvalues i k^3 a^2 j_n'(ka) h_n'(ka) (H) and
  (i k^2 a^2 / 2)(j_n h_n' + j_n' h_n) (D') from the addition theorem,
  approached under refinement.
- At the interior Dirichlet eigenvalue ka = pi of the unit sphere the plain
  equation (1/2 I - D) p = p_inc loses its conditioning while the combination
  with alpha H, alpha = i/k, keeps it, and both stay near the Mie solution.
"""
import functools

import numpy as np
import pytest
import scipy.special as sp

import oracle
from oracle import burton_miller as bm
from oracle import closed_forms as cf
from paper_1606_02383_gb300 import inputs


@functools.lru_cache(maxsize=None)
def _ops(level, k):
    V, T = inputs.icosphere(level)
    Dp, H = bm.assemble(V, T, k)
    return V, T, Dp, H


def _hn(n, x, d=False):
    return sp.spherical_jn(n, x, d) + 1j * sp.spherical_yn(n, x, d)


def _rel(A, v, lam):
    return np.linalg.norm(A @ v - lam * v) / np.linalg.norm(lam * v)


@pytest.mark.parametrize("level", [2, 3])
def test_hypersingular_annihilates_constants_at_low_k(level):
    _, _, _, H = _ops(level, 1e-9)
    assert np.abs(H.sum(axis=1)).max() < 1e-4 * np.abs(np.diag(H)).max()


def test_sphere_eigenvalues_under_refinement():
    k = 1.0
    lam_h0 = 1j * k ** 3 * sp.spherical_jn(0, k, True) * _hn(0, k, True)
    lam_d = [0.5j * k ** 2 * (sp.spherical_jn(n, k) * _hn(n, k, True) + sp.spherical_jn(n, k, True) * _hn(n, k))
             for n in (0, 1)]
    err = {}
    for level in (2, 3):
        V, T, Dp, H = _ops(level, k)
        c = oracle.geometry(V, T)[0]
        one, y1 = np.ones(len(T)), c[:, 2] / np.linalg.norm(c, axis=1)
        err[level] = (_rel(H, one, lam_h0), _rel(Dp, one, lam_d[0]), _rel(Dp, y1, lam_d[1]))
    # H on constants converges as h^2; D' as h (a factor 2 per level)
    assert err[3][0] < 5e-3 and err[2][0] / err[3][0] > 3.5
    assert err[3][1] < 0.04 and err[2][1] / err[3][1] > 1.8
    assert err[3][2] < 0.15 and err[2][2] / err[3][2] > 1.8


def test_burton_miller_keeps_its_conditioning_at_an_interior_eigenvalue():
    k = np.pi  # j_0(ka) = 0: an interior Dirichlet eigenvalue of the unit sphere
    V, T, Dp, H = _ops(3, k)
    c, _, n, _ = oracle.geometry(V, T)
    _, D = oracle.assemble(V, T, k)
    A = 0.5 * np.eye(len(T)) - D
    alpha = 1j / k
    B = A + alpha * H
    cond = lambda M: (lambda s: s[0] / s[-1])(np.linalg.svd(M, compute_uv=False))  # noqa: E731
    assert cond(A) > 50 and cond(B) < 10
    pinc = np.exp(1j * k * c[:, 2])
    p = np.linalg.solve(B, pinc - alpha * 1j * k * n[:, 2] * pinc)
    mie = cf.mie_rigid_sphere_surface(k, 1.0, c[:, 2] / np.linalg.norm(c, axis=1))
    assert np.linalg.norm(p - mie) / np.linalg.norm(mie) < 2e-2
