"""Closed forms used to pin the oracle (test infrastructure only).

All special functions come from scipy.special (library routines).  Time
convention exp(-i omega t) and G = exp(ikr)/(4 pi r) as in Section 2.1/2.3 of
the paper; the sphere's normal points out of the scatterer.
"""
from __future__ import annotations

import numpy as np
from scipy import special as sp


def _h(n, x, derivative=False):
    return sp.spherical_jn(n, x, derivative) + 1j * sp.spherical_yn(n, x, derivative)


def mie_rigid_sphere_surface(k: float, a: float, cos_theta, nmax: int | None = None):
    """Total pressure on a rigid (sound-hard) sphere of radius a for the incident
    plane wave exp(i k z):  p(a, theta) = sum_n (2n+1) i^n (i / (ka)^2) / h_n'(ka) P_n(cos theta),
    which follows from p = sum (2n+1) i^n [j_n - j_n'/h_n' h_n] P_n and the
    Wronskian j_n h_n' - j_n' h_n = i/x^2.  Sound-hard limit of the paper's
    scatterer (Section 3.3)."""
    ka = k * a
    if nmax is None:
        nmax = int(ka + 4.0 * ka ** (1.0 / 3.0) + 10)
    ct = np.asarray(cos_theta, dtype=np.float64)
    p = np.zeros(ct.shape, dtype=np.complex128)
    for n in range(nmax + 1):
        coef = (2 * n + 1) * (1j ** n) * (1j / ka ** 2) / _h(n, ka, True)
        p += coef * sp.eval_legendre(n, ct)
    return p


def mie_rigid_sphere_scattered(k: float, a: float, points, nmax: int | None = None):
    """Scattered pressure outside a rigid sphere of radius a (centred at the
    origin) for the incident plane wave exp(i k z):
    p_s(r, theta) = -sum_n (2n+1) i^n [j_n'(ka) / h_n'(ka)] h_n(kr) P_n(cos theta),
    the outgoing field (h_n = h_n^(1)) that cancels the incident field's
    normal derivative on r = a."""
    ka = k * a
    if nmax is None:
        nmax = int(ka + 4.0 * ka ** (1.0 / 3.0) + 10)
    pts = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    r = np.linalg.norm(pts, axis=1)
    ct = pts[:, 2] / r
    p = np.zeros(r.shape, dtype=np.complex128)
    for n in range(nmax + 1):
        coef = -(2 * n + 1) * (1j ** n) * sp.spherical_jn(n, ka, True) / _h(n, ka, True)
        p += coef * _h(n, k * r) * sp.eval_legendre(n, ct)
    return p


def sphere_single_layer_eigenvalue(n: int, k: float, a: float) -> complex:
    """S Y_n = i k a^2 h_n(ka) j_n(ka) Y_n on the sphere of radius a (from the
    addition theorem G = i k sum h_n(k r>) j_n(k r<) sum_m Y_nm Y_nm^*)."""
    return 1j * k * a * a * _h(n, k * a) * sp.spherical_jn(n, k * a)


def sphere_double_layer_eigenvalue(n: int, k: float, a: float) -> complex:
    """Principal value on the sphere: D Y_n = (i k^2 a^2 / 2)[j_n'(ka) h_n(ka) + h_n'(ka) j_n(ka)] Y_n
    (average of the inner and outer limits, whose difference is Y_n)."""
    ka = k * a
    return 0.5j * k * k * a * a * (sp.spherical_jn(n, ka, True) * _h(n, ka) + _h(n, ka, True) * sp.spherical_jn(n, ka))


def sphere_double_layer_static(n: int) -> float:
    """k -> 0 limit of the double-layer eigenvalue: -1/(2(2n+1))."""
    return -1.0 / (2.0 * (2 * n + 1))


def zonal_harmonic(points, n: int):
    """P_n(z / |x|): a zonal spherical harmonic of degree n (unnormalised)."""
    p = np.asarray(points, dtype=np.float64)
    return sp.eval_legendre(n, p[:, 2] / np.linalg.norm(p, axis=1))
