"""Pin of the topological derivative formula (no GPU), following the paper's own
verification (Section 3.2): the topological difference
D = (J(with a small inclusion of radius eps at x0) - J) / (4 pi eps^3 / 3)
tends to T(x0) as eps -> 0.  Here the inclusion is sound-hard and the host is
free space, so J with the inclusion is exact through the Mie series of a rigid
sphere, independent of the oracle's BEM.  This fixes c1 = 3/2, c2 = k^2 and
the adjoint convention (point sources at the observers with weights
conj(p(x_m)))."""
import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf


def _difference_and_T(k, x0, eps, c1=1.5, c2=None):
    obs = np.array([[x, y, 3.0] for x in (-1.0, 0.0, 1.0) for y in (-1.0, 0.0, 1.0)])  # 9 observers
    p_obs = np.exp(1j * k * obs[:, 2])                                                    # plane wave exp(ikz)
    J0 = 0.5 * np.sum(np.abs(p_obs) ** 2)
    x0 = np.asarray(x0, dtype=np.float64)
    # rigid sphere of radius eps at x0: the Mie field about x0, times the incident phase there
    ps = np.exp(1j * k * x0[2]) * cf.mie_rigid_sphere_scattered(k, eps, obs - x0)
    D = (0.5 * np.sum(np.abs(p_obs + ps) ** 2) - J0) / (4.0 * np.pi * eps ** 3 / 3.0)
    p0 = np.exp(1j * k * x0[2])
    gp0 = np.array([[0.0, 0.0, 1j * k * p0]])
    pa, gpa = oracle.point_source_field(x0[None], obs, np.conj(p_obs), k)
    T = oracle.topological_derivative(np.array([p0]), gp0, pa, gpa, c1, k * k if c2 is None else c2)[0]
    return D, T


@pytest.mark.parametrize("k", [1.0, 2.0])
@pytest.mark.parametrize("x0", [(0.3, -0.2, 0.5), (1.0, 0.5, -0.4), (-0.7, 0.1, 1.2)])
def test_topological_difference_converges_to_T(k, x0):
    errs = []
    for eps in (0.02, 0.01, 0.005):
        D, T = _difference_and_T(k, x0, eps / k)
        errs.append(abs(D - T) / abs(T))
    # second order in eps: each halving divides the error by about 4
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5
    assert errs[-1] < 5e-4


def test_the_pin_rejects_other_constants():
    """The same check fails for a flipped monopole sign or a wrong dipole factor."""
    for c1, c2 in ((1.5, -1.0), (3.0, 1.0), (1.0, 1.0)):
        D, T = _difference_and_T(1.0, (0.3, -0.2, 0.5), 0.005, c1=c1, c2=c2)
        assert abs(D - T) / abs(D) > 0.05
