"""Pins of the oracle's level-set update (no GPU): the Q1 matrices against
their tensor-product form and their exact properties, the decay of the
discrete sine mode in closed form, the reaction-only step, the boundary
values and the clamp."""
import numpy as np
from scipy import sparse

from oracle import levelset


def _q1_1d(n, h):
    K1 = sparse.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tolil() / h
    M1 = sparse.diags([np.ones(n - 1), 4 * np.ones(n), np.ones(n - 1)], [-1, 0, 1]).tolil() * (h / 6.0)
    K1[0, 0] = K1[-1, -1] = 1.0 / h       # end nodes belong to one element
    M1[0, 0] = M1[-1, -1] = 2.0 * h / 6.0
    return K1.tocsr(), M1.tocsr()


def test_assembly_equals_the_tensor_product_form():
    shape, h = (5, 6, 7), 0.3
    K, M = levelset.assemble(shape, h)
    (Kx, Mx), (Ky, My), (Kz, Mz) = (_q1_1d(n, h) for n in shape)
    K3 = sparse.kron(sparse.kron(Kx, My), Mz) + sparse.kron(sparse.kron(Mx, Ky), Mz) + sparse.kron(sparse.kron(Mx, My), Kz)
    M3 = sparse.kron(sparse.kron(Mx, My), Mz)
    assert abs(K - K3).max() < 1e-13 and abs(M - M3).max() < 1e-15


def test_matrices_integrate_exactly():
    shape, h = (6, 5, 4), 0.25
    K, M = levelset.assemble(shape, h)
    one = np.ones(np.prod(shape))
    assert abs(one @ (M @ one) - (5 * h) * (4 * h) * (3 * h)) < 1e-14     # the box's volume
    assert np.abs(K @ one).max() < 1e-13                                   # constants have no gradient
    x = np.indices(shape).reshape(3, -1).T * h
    lin = 0.7 * x[:, 0] - 0.2 * x[:, 1] + 1.1 * x[:, 2]
    # int |grad u|^2 for u linear = |g|^2 volume
    assert abs(lin @ (K @ lin) - (0.49 + 0.04 + 1.21) * (5 * h) * (4 * h) * (3 * h)) < 1e-12


def test_sine_mode_decays_by_the_discrete_eigenvalue():
    n = 11
    h = 1.0 / (n - 1)
    x = np.linspace(0.0, 1.0, n)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    phi = 0.5 * np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)
    zero = np.zeros_like(phi)
    dt, tau, L = 0.01, 0.3, 1.0
    new = levelset.step(phi, zero, zero, h, dt, 0.0, tau, L, 0.0)
    th = np.pi * h
    lam = 3 * (6.0 / h ** 2) * (1 - np.cos(th)) / (2 + np.cos(th))   # K v = lam M v, per axis summed
    assert np.abs(new - phi / (1.0 + dt * tau * L * L * lam)).max() < 1e-12
    # the continuous rate 3 pi^2 is approached as h^2
    assert abs(lam - 3 * np.pi ** 2) / (3 * np.pi ** 2) < 0.01


def test_reaction_step_boundary_and_clamp():
    rng = np.random.default_rng(0)
    shape, h = (6, 7, 5), 0.2
    bnd = levelset.boundary_mask(shape)
    # the boundary already holds phi_bar and F vanishes there, so with tau = 0 the
    # consistent mass cancels on both sides: M (new - phi) / dt = M F node by node
    phi = np.where(bnd, -0.5, rng.uniform(-0.9, 0.9, shape))
    To = np.where(bnd, 0.0, rng.standard_normal(shape))
    Tc = np.where(bnd, 0.0, rng.standard_normal(shape))
    dt, C = 0.05, 2.0
    new = levelset.step(phi, To, Tc, h, dt, C, 0.0, 1.0, -0.5)
    F = np.where(phi <= 0, -C * To, C * Tc)
    assert np.abs(new[~bnd] - np.clip(phi + dt * F, -1, 1)[~bnd]).max() < 1e-11
    assert np.all(new[bnd] == -0.5)
    big = levelset.step(phi, 100 * To, 100 * Tc, h, dt, C, 0.0, 1.0, -0.5)
    assert big.min() == -1.0 and big.max() == 1.0
