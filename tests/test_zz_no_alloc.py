"""bem_apply_noalloc: the apply for callers that cannot allocate device memory.

Such callers (a program whose memory pool already owns the whole GPU, or a
latency-critical loop that must stay out of the driver's allocation path) get
the same operator with the per-call scratch in a fixed library array.  This
test calls the entry point through the C ABI twice in a row and checks each
result against bem_apply on the same handle.  It lives in its own file,
collected last, and passes alone or after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1606_02383_gb300 import _lib, inputs
from paper_1606_02383_gb300.operator import Operator

pytestmark = pytest.mark.gpu


def _noalloc(op, x, y, z):
    lib = _lib.load()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.bem_apply_noalloc(op._h, x.shape[0], _lib.BEM_C128, x.data_ptr(), y.data_ptr(), z.data_ptr(), 0, s)


@pytest.mark.parametrize("mode,p,leaf", [("mixed", 10, 3), ("fp64", 8, 2), ("direct64", 0, 0)])
def test_noalloc_matches_apply_twice(cuda_ok, mode, p, leaf):
    V, T = inputs.icosphere(3)
    n = T.shape[0]
    op = Operator(V, T, 1.0, p=p, mode=mode, leaf_level=leaf)
    for call in range(2):
        x = torch.from_numpy(inputs.random_density(n, 2, seed=call, stream=0)).cuda()
        y = torch.from_numpy(inputs.random_density(n, 2, seed=call, stream=1)).cuda()
        ref = op.apply(x, y).cpu().numpy()
        z = torch.full((2, n), float("nan"), dtype=torch.complex128, device="cuda")
        _lib.check(_noalloc(op, x, y, z))
        got = z.cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 1e-6, (mode, call, err)


def test_noalloc_rejects_oversized_calls(cuda_ok):
    V, T = inputs.icosphere(6)  # 81,920 triangles
    n = T.shape[0]
    op = Operator(V, T, 1.0, p=0, eps=1e-5, mode="mixed", max_nrhs=16)
    x = torch.zeros((16, n), dtype=torch.complex128, device="cuda")
    z = torch.empty_like(x)
    rc = _noalloc(op, x, x, z)
    assert rc == _lib.BEM_ERR_INVALID_ARG
    assert b"scratch bytes" in _lib.load().bem_last_error()
    # a right-hand side count above the handle's max_nrhs is rejected like
    # bem_apply rejects it, even where the scratch would fit
    V, T = inputs.icosphere(2)
    n = T.shape[0]
    op = Operator(V, T, 1.0, p=8, mode="mixed", leaf_level=2, max_nrhs=2)
    x = torch.zeros((3, n), dtype=torch.complex128, device="cuda")
    z = torch.empty_like(x)
    rc = _noalloc(op, x, x, z)
    assert rc == _lib.BEM_ERR_INVALID_ARG
    assert b"max_nrhs" in _lib.load().bem_last_error()
