"""The level-set boundary by marching tetrahedra on the GPU vs the oracle:
vertex and triangle indices bit-exact (the output order is part of the
definition), positions to 1e-14 (both sides use the same unfused IEEE
operations)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1606_02383_gb300 import _lib, inputs
from paper_1606_02383_gb300.operator import isosurface

pytestmark = pytest.mark.gpu


def _compare(phi, lo, h, t):
    V, T = isosurface(torch.from_numpy(phi), lo, h, t)
    Vr, Tr = oracle.isosurface(phi, lo, h, t)
    V, T = V.cpu().numpy(), T.cpu().numpy()
    assert V.shape == Vr.shape and T.shape == Tr.shape
    assert np.array_equal(T, Tr)
    if len(V):
        assert np.abs(V - Vr).max() <= 1e-14
    return V, T


def test_level_set_surface_of_the_differentiation_workload(cuda_ok):
    phi, lo, h = inputs.level_set_function(0, 20, 64)
    t = inputs.level_set_level()
    V, T = _compare(phi, lo, h, t)
    assert T.shape == (30004, 3)


@pytest.mark.parametrize("shape", [(5, 7, 9), (3, 2, 4), (2, 2, 2), (17, 33, 9)])
@pytest.mark.parametrize("seed", [0, 1])
def test_ragged_grids(cuda_ok, shape, seed):
    rng = np.random.default_rng([seed, 11])
    phi = rng.standard_normal(shape)
    _compare(phi, (-0.3, 0.2, 1.0), 0.37, 0.1)


def test_empty_levels(cuda_ok):
    phi = np.random.default_rng(3).standard_normal((6, 5, 4))
    for t in (10.0, -10.0):
        V, T = _compare(phi, (0.0, 0.0, 0.0), 1.0, t)
        assert V.shape == (0, 3) and T.shape == (0, 3)


def test_capacity_and_nan_errors(cuda_ok):
    lib = _lib.load()
    phi = torch.from_numpy(np.random.default_rng(4).standard_normal((6, 6, 6))).cuda()
    lo = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    counts = (ctypes.c_int64 * 2)()
    V = torch.empty((1, 3), dtype=torch.float64, device="cuda")
    T = torch.empty((1, 3), dtype=torch.int32, device="cuda")
    rc = lib.bem_isosurface(6, 6, 6, phi.data_ptr(), lo, 1.0, 0.0, V.data_ptr(), 1, T.data_ptr(), 1, counts,
                            torch.cuda.current_stream().cuda_stream)
    assert rc == _lib.BEM_ERR_INVALID_ARG and counts[0] > 1 and counts[1] > 1
    Vr, Tr = oracle.isosurface(phi.cpu().numpy(), (0.0, 0.0, 0.0), 1.0, 0.0)
    assert (counts[0], counts[1]) == Vr.shape[:1] + Tr.shape[:1]
    bad = phi.clone()
    bad[2, 3, 1] = float("nan")
    with pytest.raises(_lib.BemError) as e:
        isosurface(bad, (0.0, 0.0, 0.0), 1.0, 0.0)
    assert e.value.code == _lib.BEM_ERR_NUMERIC
