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


def _jn_derivs(n, x):
    """j_n(x), j_n'(x), j_n''(x) (the last from the spherical Bessel equation)."""
    j = sp.spherical_jn(n, x)
    jp = sp.spherical_jn(n, x, True)
    jpp = -2.0 / x * jp - (1.0 - n * (n + 1) / (x * x)) * j
    return j, jp, jpp


def elastic_sphere_coefficients(n: int, omega: float, a: float, lam: float, mu: float, rho_s: float,
                                rho_f: float, c_f: float):
    """(A_n, B_n, C_n) of the plane wave exp(i k z), k = omega / c_f, scattered by
    an isotropic elastic sphere of radius a in the fluid (Section 2.1's coupled
    problem with the boundary conditions t = -p n and dp/dn = rho_f omega^2 u.n,
    n out of the sphere):
      fluid   p = sum_n [(2n+1) i^n j_n(kr) + A_n h_n(kr)] P_n(cos theta),
      solid   u = grad phi + curl curl (r chi),  phi = sum B_n j_n(k_L r) P_n,
              chi = sum C_n j_n(k_T r) P_n,  k_L = omega / c_L, k_T = omega / c_T,
              c_L^2 = (lambda + 2 mu) / rho_s, c_T^2 = mu / rho_s.
    With f = j_n(k_L r), g = j_n(k_T r), the solid's fields per order are
      u_r     = B k_L f' + C n(n+1) g / r,
      u_theta = [B f / r + C (r g)' / r] dP_n/dtheta,
      sigma_rr = B (-lambda k_L^2 f + 2 mu k_L^2 f'') + 2 mu C n(n+1) (g / r)',
      sigma_r_theta = mu [u_r / r + d u_theta / dr - u_theta / r] (per dP_n/dtheta),
    and at r = a: sigma_rr = -p, sigma_r_theta = 0, dp/dr = rho_f omega^2 u_r.
    Order 0 has no shear part (C_0 = 0)."""
    k = omega / c_f
    kl = omega * np.sqrt(rho_s / (lam + 2.0 * mu))
    kt = omega * np.sqrt(rho_s / mu)
    ka, xl, xt = k * a, kl * a, kt * a
    inc = (2 * n + 1) * (1j ** n)
    f, fp, fpp = _jn_derivs(n, xl)
    g, gp, gpp = _jn_derivs(n, xt)
    nn = n * (n + 1)
    # u_r coefficients and their r-derivatives at r = a
    F1, F2 = kl * fp, nn * g / a
    F1p, F2p = kl * kl * fpp, nn * (kt * gp / a - g / (a * a))
    # u_theta coefficients G1 = f / r, G2 = (g + r g') / r and their r-derivatives
    G1, G2 = f / a, (g + xt * gp) / a
    G1p = kl * fp / a - f / (a * a)
    G2p = kt * gp / a - g / (a * a) + kt * kt * gpp
    s1 = -lam * kl * kl * f + 2.0 * mu * F1p
    s2 = 2.0 * mu * F2p
    t1 = mu * (F1 / a + G1p - G1 / a)
    t2 = mu * (F2 / a + G2p - G2 / a)
    h, hp = _h(n, ka), _h(n, ka, True)
    beta = rho_f * omega * omega
    if n == 0:
        M = np.array([[h, s1], [k * hp, -beta * F1]], dtype=np.complex128)
        rhs = np.array([-inc * sp.spherical_jn(0, ka), -inc * k * sp.spherical_jn(0, ka, True)])
        A, B = np.linalg.solve(M, rhs)
        return A, B, 0.0
    M = np.array([[h, s1, s2], [0.0, t1, t2], [k * hp, -beta * F1, -beta * F2]], dtype=np.complex128)
    rhs = np.array([-inc * sp.spherical_jn(n, ka), 0.0, -inc * k * sp.spherical_jn(n, ka, True)])
    A, B, C = np.linalg.solve(M, rhs)
    return A, B, C


def elastic_sphere_surface(omega: float, a: float, lam: float, mu: float, rho_s: float, rho_f: float, c_f: float,
                           cos_theta, nmax: int | None = None):
    """Total pressure on the fluid side of the elastic sphere's surface for the
    plane wave exp(i k z), p(a, theta) = sum_n [(2n+1) i^n j_n(ka) + A_n h_n(ka)] P_n."""
    k = omega / c_f
    ka = k * a
    if nmax is None:
        nmax = int(ka + 4.0 * ka ** (1.0 / 3.0) + 12)
    ct = np.asarray(cos_theta, dtype=np.float64)
    p = np.zeros(ct.shape, dtype=np.complex128)
    for n in range(nmax + 1):
        A, _, _ = elastic_sphere_coefficients(n, omega, a, lam, mu, rho_s, rho_f, c_f)
        p += ((2 * n + 1) * (1j ** n) * sp.spherical_jn(n, ka) + A * _h(n, ka)) * sp.eval_legendre(n, ct)
    return p


def fluid_sphere_coefficient(n: int, omega: float, a: float, bulk_in: float, rho_in: float, rho_f: float,
                             c_f: float):
    """A_n of the plane wave scattered by a fluid sphere (bulk modulus bulk_in,
    density rho_in): pressure and (1 / rho) dp/dr continuous at r = a."""
    k = omega / c_f
    ki = omega * np.sqrt(rho_in / bulk_in)
    ka, kia = k * a, ki * a
    inc = (2 * n + 1) * (1j ** n)
    ji, jip = sp.spherical_jn(n, kia), sp.spherical_jn(n, kia, True)
    # inc j + A h = D ji ;  (inc k j' + A k h') / rho_f = D ki ji' / rho_in
    M = np.array([[_h(n, ka), -ji], [k * _h(n, ka, True) / rho_f, -ki * jip / rho_in]], dtype=np.complex128)
    rhs = np.array([-inc * sp.spherical_jn(n, ka), -inc * k * sp.spherical_jn(n, ka, True) / rho_f])
    A, _ = np.linalg.solve(M, rhs)
    return A
