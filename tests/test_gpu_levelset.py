"""One step of the level-set update on the GPU (bem_levelset_step) against the
oracle's step (Section 2.4: Q1 on the voxels, implicit diffusion, explicit
topological-derivative term, phi_bar on the box boundary, clamp to [-1, 1]).

Both sides solve the interior system by conjugate gradients to a relative
residual of 1e-13 (the oracle with scipy on its assembled matrices, the GPU
matrix-free on the 27-point stencil), so the steps agree to 1e-10.
"""
import numpy as np
import pytest
import torch

from oracle import levelset
from paper_1606_02383_gb300 import _lib
from paper_1606_02383_gb300.operator import levelset_step

pytestmark = pytest.mark.gpu


def _fields(shape, seed):
    rng = np.random.default_rng(seed)
    idx = np.indices(shape).astype(np.float64)
    c = np.array(shape, dtype=np.float64)[:, None, None, None] / 2.0
    r = np.sqrt(((idx - c) ** 2).sum(axis=0)) / (min(shape) / 2.0)
    phi = np.clip(0.8 - 1.2 * r + 0.1 * rng.standard_normal(shape), -1.0, 1.0)
    To = rng.standard_normal(shape)
    Tc = rng.standard_normal(shape)
    return phi, To, Tc


@pytest.mark.parametrize("shape,h,dt,C,tau,L,phi_bar", [
    ((13, 11, 9), 0.1, 0.02, 0.5, 0.4, 1.0, -0.5),
    ((20, 20, 20), 0.05, 0.005, 2.0, 1.0, 0.5, -1.0),
    ((7, 16, 5), 0.3, 0.1, 0.0, 2.0, 2.0, -0.2),      # diffusion alone
    ((9, 8, 10), 0.2, 0.05, 1.0, 0.0, 1.0, -0.5),     # reaction alone (tau = 0)
])
def test_step_matches_oracle(cuda_ok, shape, h, dt, C, tau, L, phi_bar):
    phi, To, Tc = _fields(shape, seed=sum(shape))
    ref = levelset.step(phi, To, Tc, h, dt, C, tau, L, phi_bar)
    out, iters, rel = levelset_step(torch.from_numpy(phi), torch.from_numpy(To), torch.from_numpy(Tc), h, dt, C, tau,
                                    L, phi_bar)
    got = out.cpu().numpy()
    assert rel <= 1e-13
    assert np.abs(got - ref).max() <= 1e-10, np.abs(got - ref).max()
    bnd = levelset.boundary_mask(shape)
    assert np.all(got[bnd] == np.clip(phi_bar, -1, 1))
    assert got.min() >= -1.0 and got.max() <= 1.0


def test_lattice_without_interior_and_errors(cuda_ok):
    phi, To, Tc = _fields((2, 6, 5), seed=3)
    out, iters, rel = levelset_step(torch.from_numpy(phi), torch.from_numpy(To), torch.from_numpy(Tc), 0.1, 0.01, 1.0,
                                    0.5, 1.0, -0.4)
    assert iters == 0 and np.all(out.cpu().numpy() == -0.4)
    with pytest.raises(_lib.BemError):
        levelset_step(torch.from_numpy(phi), torch.from_numpy(To), torch.from_numpy(Tc), 0.0, 0.01, 1.0, 0.5, 1.0, -0.4)
    # too few iterations: not converged, the last iterate is returned when asked
    phi, To, Tc = _fields((24, 24, 24), seed=4)
    out, iters, rel = levelset_step(torch.from_numpy(phi), torch.from_numpy(To), torch.from_numpy(Tc), 0.05, 0.5, 1.0,
                                    1.0, 1.0, -0.5, max_iter=2, raise_on_fail=False)
    assert iters == 2 and rel > 1e-13
    with pytest.raises(_lib.BemError) as e:
        levelset_step(torch.from_numpy(phi), torch.from_numpy(To), torch.from_numpy(Tc), 0.05, 0.5, 1.0, 1.0, 1.0, -0.5,
                      max_iter=2)
    assert e.value.code == _lib.BEM_ERR_NOT_CONVERGED
