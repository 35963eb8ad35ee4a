"""Pins of the FP64 CPU oracle against things other than itself.

Each test names what fixes the expected value: a closed form (sphere
eigenvalues, Mie series), an identity (Gauss, reciprocity), a library routine
(numpy.linalg.solve, scipy adaptive quadrature), or brute force.
"""
import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle import closed_forms as cf
from paper_1606_02383_gb300 import inputs


@pytest.fixture(scope="module")
def sphere3():
    return inputs.icosphere(3)


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


# --- self term: closed form + polar remainder vs 2-D adaptive quadrature ------

def _self_adaptive(V, k):
    """int_T exp(ikr)/(4 pi r) dA at the centroid, by scipy's adaptive dblquad in
    polar coordinates about the centroid (the 1/r cancels the Jacobian)."""
    c = V.mean(axis=0)
    e1 = V[1] - V[0]
    nrm = np.cross(e1, V[2] - V[0])
    nrm /= np.linalg.norm(nrm)
    u = e1 / np.linalg.norm(e1)
    w = np.cross(nrm, u)
    P = np.array([[(v - c) @ u, (v - c) @ w] for v in V])
    tot = 0.0 + 0.0j
    for e in range(3):
        A, B = P[e], P[(e + 1) % 3]
        ta, tb = np.arctan2(A[1], A[0]), np.arctan2(B[1], B[0])
        if tb < ta:
            tb += 2 * np.pi
        d = B - A

        def rmax(t):
            uu = np.array([np.cos(t), np.sin(t)])
            # solve rho*uu = A + s*d
            M = np.array([[uu[0], -d[0]], [uu[1], -d[1]]])
            return np.linalg.solve(M, A)[0]

        re = integrate.dblquad(lambda r, t: np.cos(k * r) / (4 * np.pi), ta, tb, 0.0, rmax, epsabs=1e-14, epsrel=1e-13)[0]
        im = integrate.dblquad(lambda r, t: np.sin(k * r) / (4 * np.pi), ta, tb, 0.0, rmax, epsabs=1e-14, epsrel=1e-13)[0]
        tot += re + 1j * im
    return tot


@pytest.mark.parametrize("k", [0.0, 1.0, 7.5])
def test_self_term_matches_adaptive_quadrature(k):
    rng = np.random.default_rng(3)
    slivers = [np.array([[0.0, 0, 0], [0.2, 0, 0], [0.1, 0.002, 0.0]]),           # aspect ~ 1e-2
               np.array([[0.0, 0, 0], [0.05, 0.001, 0.0005], [0.3, 0.0, 0.0]])]   # long and thin
    for V in [rng.normal(size=(3, 3)) * 0.3 for _ in range(3)] + slivers:
        T = np.array([[0, 1, 2]], dtype=np.int32)
        s, d = oracle.entries(V, T, k, [0], [0])
        ref = _self_adaptive(V, k)
        assert abs(s[0] - ref) <= 1e-11 * abs(ref), (s[0], ref)
        assert d[0] == 0.0


# --- single layer: sphere eigenvalues (closed form), O(h^2) convergence ------

@pytest.mark.parametrize("k", [1.0, 3.0])
def test_single_layer_sphere_eigenvalues_converge(k):
    errs = []
    for lev in (2, 3):
        V, T = inputs.icosphere(lev)
        c, _, _, _ = oracle.geometry(V, T)
        e = []
        for n in (0, 1, 2):
            yn = cf.zonal_harmonic(c, n)[None, :].astype(complex)
            z = oracle.apply(V, T, k, y=yn)[0]
            lam = cf.sphere_single_layer_eigenvalue(n, k, 1.0)
            e.append(np.linalg.norm(z - lam * yn[0]) / np.linalg.norm(yn[0]))
        errs.append(max(e))
    assert errs[1] < 0.01
    assert errs[0] / errs[1] > 2.5  # observed order >= ~1.3 per halving of h


@pytest.mark.parametrize("k", [1.0, 3.0])
def test_double_layer_sphere_eigenvalues_converge(k):
    errs = []
    for lev in (2, 3):
        V, T = inputs.icosphere(lev)
        c, _, _, _ = oracle.geometry(V, T)
        e = []
        for n in (0, 1, 2):
            xn = cf.zonal_harmonic(c, n)[None, :].astype(complex)
            z = -oracle.apply(V, T, k, x=xn, flags=oracle.FLAG_NO_HALF)[0]   # = D x
            lam = cf.sphere_double_layer_eigenvalue(n, k, 1.0)
            e.append(np.linalg.norm(z - lam * xn[0]) / np.linalg.norm(xn[0]))
        errs.append(max(e))
    assert errs[1] < 0.0025 * (1.0 + k * k)   # discretisation error grows like (k h)^2
    assert errs[0] / errs[1] > 2.5


def test_double_layer_static_limit_eigenvalues(sphere3):
    V, T = sphere3
    c, _, _, _ = oracle.geometry(V, T)
    for n in (0, 1, 3):
        xn = cf.zonal_harmonic(c, n)[None, :].astype(complex)
        z = -oracle.apply(V, T, 0.0, x=xn, flags=oracle.FLAG_NO_HALF)[0]
        assert np.linalg.norm(z - cf.sphere_double_layer_static(n) * xn[0]) / np.linalg.norm(xn[0]) < 5e-3


# --- Gauss identity for the double layer at k = 0 ---------------------------

def test_gauss_identity(sphere3):
    V, T = sphere3
    nt = T.shape[0]
    ones = np.ones((1, nt), complex)
    on = -oracle.apply(V, T, 0.0, x=ones, flags=oracle.FLAG_NO_HALF)[0]       # D 1 at centroids
    assert np.max(np.abs(on + 0.5)) < 1e-4
    # with the 1/2 term: (1/2 I - D) 1 = 1 on the surface
    assert np.max(np.abs(oracle.apply(V, T, 0.0, x=ones)[0] - 1.0)) < 1e-4
    pts_in = np.array([[0.0, 0.0, 0.0], [0.3, -0.2, 0.1], [0.0, 0.5, -0.5]])
    pts_out = np.array([[2.0, 0.0, 0.0], [1.5, 1.5, -1.0], [0.0, 0.0, -3.0]])
    w_in = -oracle.eval_points(V, T, 0.0, pts_in, x=ones)[0]    # = sum_j D(p, j)
    w_out = -oracle.eval_points(V, T, 0.0, pts_out, x=ones)[0]
    assert np.max(np.abs(w_in + 1.0)) < 2e-5    # quadrature error of R_0 at distance ~h/0.1
    assert np.max(np.abs(w_out)) < 1e-6


# --- reciprocity of the single-layer kernel (1-point centroid rule) ---------

def test_single_layer_reciprocity():
    V, T = inputs.icosphere(2)
    _, area, _, _ = oracle.geometry(V, T)
    rng = np.random.default_rng(7)
    ii = rng.integers(0, T.shape[0], 200)
    jj = rng.integers(0, T.shape[0], 200)
    keep = ii != jj
    ii, jj = ii[keep], jj[keep]
    k = 2.0
    sij, dij = oracle.entries(V, T, k, ii, jj, flags=oracle.FLAG_RULE1)
    sji, dji = oracle.entries(V, T, k, jj, ii, flags=oracle.FLAG_RULE1)
    np.testing.assert_allclose(sij / area[jj], sji / area[ii], rtol=1e-13)
    # the double layer is not symmetric: a transposed operand would make it so
    assert np.max(np.abs(dij / area[jj] - dji / area[ii])) > 1e-3


# --- dense LU vs numpy.linalg.solve ----------------------------------------

def test_lu_matches_numpy(sphere3):
    V, T = sphere3
    k = 1.0
    S, D = oracle.assemble(V, T, k)
    A = 0.5 * np.eye(T.shape[0]) - D + 0.3 * S
    b = inputs.random_density(T.shape[0], 2, seed=1)
    x = oracle.lu_solve(A, b)
    ref = np.linalg.solve(A, b.T).T
    assert _rel(x, ref) < 1e-12


# --- apply/assemble/adjoint consistency (loops and conjugation) --------------

def test_apply_adjoint_dot_product(sphere3):
    V, T = sphere3
    k = 2.0
    nt = T.shape[0]
    x = inputs.random_density(nt, 1, seed=2)
    y = inputs.random_density(nt, 1, seed=3)
    g = inputs.random_density(nt, 1, seed=4)
    z = oracle.apply(V, T, k, x=x, y=y)
    gx, gy = oracle.adjoint(V, T, k, g)
    lhs = np.vdot(g, z)
    rhs = np.vdot(gx, x) + np.vdot(gy, y)
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(z) * np.linalg.norm(g)
    S, D = oracle.assemble(V, T, k)
    z2 = (0.5 * x[0] - D @ x[0] + S @ y[0])
    assert _rel(z[0], z2) < 1e-14


# --- Mie series for the rigid sphere (the sound-hard limit, Section 3.3) ------

def test_mie_rigid_sphere_solution_converges():
    k = 1.0
    errs = []
    for lev in (2, 3):
        V, T = inputs.icosphere(lev)
        c, _, _, _ = oracle.geometry(V, T)
        S, D = oracle.assemble(V, T, k)
        A = 0.5 * np.eye(T.shape[0]) - D
        b = inputs.plane_wave(c, k)[None, :]
        p = oracle.lu_solve(A, b)[0]
        ref = cf.mie_rigid_sphere_surface(k, 1.0, c[:, 2] / np.linalg.norm(c, axis=1))
        errs.append(_rel(p, ref))
    assert errs[1] < 5e-3
    assert errs[0] / errs[1] > 2.5


def test_mie_series_truncation_independent():
    ct = np.linspace(-1, 1, 17)
    a = cf.mie_rigid_sphere_surface(5.0, 1.0, ct)
    b = cf.mie_rigid_sphere_surface(5.0, 1.0, ct, nmax=60)
    assert np.max(np.abs(a - b)) < 1e-10 * np.max(np.abs(b))


def test_mie_scattered_field_meets_surface_formula():
    """On r = a the incident plus scattered closed form equals the surface
    closed form (the latter simplified through the Wronskian, the former not)."""
    for k in (0.7, 3.0, 8.0):
        th = np.linspace(0.05, np.pi - 0.05, 23)
        pts = np.stack([np.sin(th), 0 * th, np.cos(th)], axis=1)
        tot = np.exp(1j * k * pts[:, 2]) + cf.mie_rigid_sphere_scattered(k, 1.0, pts)
        assert _rel(tot, cf.mie_rigid_sphere_surface(k, 1.0, np.cos(th))) < 1e-11


def test_offsurface_double_layer_of_the_mie_pressure_is_the_scattered_field():
    """For a rigid body the exterior representation formula reduces to
    p_s(x) = (D p)(x), the double layer with the normals pointing into the
    fluid (its exterior limit D p + p/2 turns p = p_inc + D p into the surface
    equation (1/2 I - D) p = p_inc).  The oracle's off-surface evaluation,
    which returns S y - D x, of the exact Mie surface pressure reproduces the
    Mie scattered field outside the sphere to the discretisation error, which
    falls as h^2."""
    k = 2.0
    rng = np.random.default_rng(3)
    d = rng.normal(size=(24, 3))
    pts = d / np.linalg.norm(d, axis=1, keepdims=True) * rng.uniform(1.5, 3.0, size=(24, 1))
    ref = cf.mie_rigid_sphere_scattered(k, 1.0, pts)
    errs = []
    for lev in (3, 4):
        V, T = inputs.icosphere(lev)
        c, _, _, _ = oracle.geometry(V, T)
        p = cf.mie_rigid_sphere_surface(k, 1.0, c[:, 2] / np.linalg.norm(c, axis=1))[None, :]
        ps = -oracle.eval_points(V, T, k, pts, x=p)[0]  # -(S y - D x) with y = 0, x = p
        errs.append(_rel(ps, ref))
    assert errs[1] < 1e-2
    assert errs[0] / errs[1] > 2.5


def test_offsurface_gradient_matches_central_differences():
    """grad_p of the off-surface field against central differences of the
    (pinned) field itself, for both layers, at points where every rule R_0,
    R_1, R_2 applies (the rule changes only across the 2h / 4h thresholds,
    which the tiny steps do not cross)."""
    V, T = inputs.icosphere(2)
    n, k = T.shape[0], 2.5
    x = inputs.random_density(n, 1, seed=6, stream=0)
    y = inputs.random_density(n, 1, seed=6, stream=1)
    c, _, _, _ = oracle.geometry(V, T)
    nrm = c / np.linalg.norm(c, axis=1, keepdims=True)
    pts = np.concatenate([c[[3, 40, 77]] + nrm[[3, 40, 77]] * np.array([[0.13], [0.45], [0.9]]),
                          np.array([[0.2, -0.1, 0.3], [2.0, 1.0, -0.5]])])
    g = oracle.eval_points_grad(V, T, k, pts, x=x, y=y)[0]
    h = 1e-5
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fd = (oracle.eval_points(V, T, k, pts + e, x=x, y=y)[0] - oracle.eval_points(V, T, k, pts - e, x=x, y=y)[0]) / (2 * h)
        assert np.max(np.abs(fd - g[:, a])) < 1e-6 * np.max(np.abs(g)), a


def test_offsurface_gradient_of_the_mie_field():
    """grad p_s of the rigid sphere (D p of the exact Mie surface pressure)
    against the gradient of the Mie scattered-field closed form (central
    differences of the series), to the discretisation error."""
    k = 2.0
    rng = np.random.default_rng(8)
    d = rng.normal(size=(12, 3))
    pts = d / np.linalg.norm(d, axis=1, keepdims=True) * rng.uniform(1.5, 2.5, size=(12, 1))
    h = 1e-5
    ref = np.stack([(cf.mie_rigid_sphere_scattered(k, 1.0, pts + h * np.eye(3)[a]) -
                     cf.mie_rigid_sphere_scattered(k, 1.0, pts - h * np.eye(3)[a])) / (2 * h) for a in range(3)], axis=1)
    V, T = inputs.icosphere(4)
    c, _, _, _ = oracle.geometry(V, T)
    p = cf.mie_rigid_sphere_surface(k, 1.0, c[:, 2] / np.linalg.norm(c, axis=1))[None, :]
    g = -oracle.eval_points_grad(V, T, k, pts, x=p)[0]
    assert _rel(g, ref) < 1e-2


# --- vertex / wavenumber gradient (forward-mode duals over every entry) ------

def _loss(V, T, k, g, x, y):
    """L = sum Re(conj(g) z), z = (1/2 I - D) x + S y: the loss whose upstream gradient is g."""
    z = oracle.apply(V, T, k, x, y)
    return float(np.sum((np.conj(g) * z).real))


def _grad_case(mesh, k, nrhs=2, seed=5):
    V, T = mesh
    nt = T.shape[0]
    rng = np.random.default_rng(seed)
    draw = lambda: rng.standard_normal((nrhs, nt)) + 1j * rng.standard_normal((nrhs, nt))
    return V, T, k, draw(), draw(), draw()


def _jittered_icosphere():
    V, T = inputs.icosphere(1)
    rng = np.random.default_rng(3)
    return V * (1.0 + 0.08 * rng.standard_normal((V.shape[0], 1))), T


@pytest.mark.parametrize("which", ["icosphere1_jittered", "level_set_slivers"])
def test_gradient_matches_central_differences(which):
    """Pin: the derivative is the limit of the difference quotient of the pinned
    apply.  Coarse meshes put most pairs inside the refined rules R_1, R_2 and
    every self term on the path; the level-set mesh adds sliver triangles."""
    mesh = _jittered_icosphere() if which == "icosphere1_jittered" else inputs.level_set_mesh(seed=1, grid=16, target=300)
    V, T, k, g, x, y = _grad_case(mesh, 2.3)
    dV, dk = oracle.grad(V, T, k, g, x, y)
    h = 1e-6
    rng = np.random.default_rng(11)
    for v in rng.choice(V.shape[0], 6, replace=False):
        for d in range(3):
            Vp, Vm = V.copy(), V.copy()
            Vp[v, d] += h
            Vm[v, d] -= h
            fd = (_loss(Vp, T, k, g, x, y) - _loss(Vm, T, k, g, x, y)) / (2 * h)
            assert abs(dV[v, d] - fd) <= 1e-6 * max(1.0, abs(fd)), (v, d, dV[v, d], fd)
    fdk = (_loss(V, T, k + h, g, x, y) - _loss(V, T, k - h, g, x, y)) / (2 * h)
    assert abs(dk - fdk) <= 1e-6 * max(1.0, abs(fdk))


@pytest.mark.parametrize("sliver", [False, True])
def test_self_term_gradient_matches_central_differences(sliver):
    """One triangle: L = Re(conj(g) S_11 y) is the exact self term alone (D_11 = 0)."""
    V = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.3, 0.8, 0.2]])
    if sliver:
        V[2] = [0.5, 0.03, 0.01]
    T = np.array([[0, 1, 2]], dtype=np.int32)
    g, x, y = np.array([[0.7 - 0.4j]]), np.array([[0.3 + 0.9j]]), np.array([[1.1 + 0.2j]])
    k = 4.0
    dV, dk = oracle.grad(V, T, k, g, x, y)
    h = 1e-6
    for v in range(3):
        for d in range(3):
            Vp, Vm = V.copy(), V.copy()
            Vp[v, d] += h
            Vm[v, d] -= h
            fd = (_loss(Vp, T, k, g, x, y) - _loss(Vm, T, k, g, x, y)) / (2 * h)
            assert abs(dV[v, d] - fd) <= 1e-7 * max(1.0, abs(fd)), (v, d, dV[v, d], fd)
    fdk = (_loss(V, T, k + h, g, x, y) - _loss(V, T, k - h, g, x, y)) / (2 * h)
    assert abs(dk - fdk) <= 1e-7 * max(1.0, abs(fdk))


def test_gradient_invariances_and_scaling_identity():
    """Pins from the symmetries of the operator, exact for the rule-defined entries:
    - translating the mesh changes no entry: sum_v dL/dV_v = 0;
    - rotating it changes none: sum_v V_v x dL/dV_v = 0;
    - scaling: S(lam V, k) = lam S(V, lam k) and D(lam V, k) = D(V, lam k), so
      sum_v V_v . dL/dV_v = Re<g, S y> + k dL/dk."""
    V, T, k, g, x, y = _grad_case(inputs.level_set_mesh(seed=2, grid=16, target=300), 3.1)
    V = V + np.array([0.4, -0.2, 0.9])  # away from the origin, so rotation and scaling are not trivial
    dV, dk = oracle.grad(V, T, k, g, x, y)
    scale = np.abs(V).sum(axis=1) @ np.abs(dV).sum(axis=1)
    assert np.abs(dV.sum(axis=0)).max() <= 1e-12 * np.abs(dV).sum()
    assert np.abs(np.cross(V, dV).sum(axis=0)).max() <= 1e-12 * scale
    sy = float(np.sum((np.conj(g) * oracle.apply(V, T, k, None, y)).real))
    assert abs(np.sum(V * dV) - (sy + k * dk)) <= 1e-12 * scale


def test_gradient_of_selected_vertices_equals_full():
    V, T, k, g, x, y = _grad_case(_jittered_icosphere(), 1.7)
    dV, _ = oracle.grad(V, T, k, g, x, y)
    sel = np.array([0, 7, 33, 41])
    dVs, dks = oracle.grad(V, T, k, g, x, y, vertices=sel)
    assert dks is None
    np.testing.assert_allclose(dVs, dV[sel], rtol=1e-13, atol=1e-13 * np.abs(dV).max())
