"""Topological derivative of the observation objective, written out (test
infrastructure only: only the tests, the smoke check and the bench's CPU leg
use it).

Section 2.5 (with the sound-hard limit of the inclusion's constants): for
f = 1/2 sum_m |p(x_m)|^2 the adjoint field is the field of point sources at the
observers with weights conj(p(x_m)) (plus its scattered part when a scatterer
is present), and

    T(x) = Re[c1 grad p(x) . grad pa(x) - c2 p(x) pa(x)],

c1 = 3 (rho_s - rho_f) / (2 rho_s + rho_f) and c2 = rho_f omega^2 (Lambda_s -
Lambda_f) / (Lambda_s Lambda_f) for an elastic inclusion; the sound-hard
(rigid, rho_s -> inf, Lambda_s -> inf) limit in units rho_f = c_f = 1 is
c1 = 3/2, c2 = k^2.
"""
from __future__ import annotations

import numpy as np


def point_source_field(points, sources, weights, k):
    """u(x) = sum_m w_m G(x - x_m) and grad u, G = exp(ikr) / (4 pi r)."""
    x = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    s = np.asarray(sources, dtype=np.float64).reshape(-1, 3)
    w = np.asarray(weights, dtype=np.complex128).reshape(-1)
    d = x[:, None, :] - s[None, :, :]
    r = np.linalg.norm(d, axis=2)
    e = np.exp(1j * k * r) * w[None, :]
    u = np.sum(e / (4.0 * np.pi * r), axis=1)
    # grad G(x - x_m) = exp(ikr) (ikr - 1) / (4 pi r^3) (x - x_m)
    gu = np.einsum("pm,pmc->pc", e * (1j * k * r - 1.0) / (4.0 * np.pi * r ** 3), d)
    return u, gu


def topological_derivative(p, grad_p, pa, grad_pa, c1, c2):
    """T = Re[c1 grad p . grad pa - c2 p pa] pointwise."""
    return np.real(c1 * np.sum(np.asarray(grad_p) * np.asarray(grad_pa), axis=-1) - c2 * np.asarray(p) * np.asarray(pa))
