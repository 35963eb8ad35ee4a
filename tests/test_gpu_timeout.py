"""The bounded-wait path of the tensor-core translations.

Every mbarrier wait in the translation kernel gives up after a bounded number
of SM clocks; the CTA then flags the expiry, waits (bounded) for its own copies
and MMAs, frees its tensor memory and returns, and the host reports
BEM_ERR_TIMEOUT.  Here the wait is made to run out without any fault: the
diagnostic hook withholds every CTA's first matrix copy (so nothing is in
flight) and bounds the first wait at 2^14 clocks.  The same handle must then
apply correctly again.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1606_02383_gb300 import _lib, inputs
from paper_1606_02383_gb300.operator import Operator

pytestmark = pytest.mark.gpu


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("pipeline", [1, 2, 3, 4])
def test_expired_wait_reports_timeout_and_handle_recovers(cuda_ok, pipeline):
    """Every translation loop (block-synchronous, warp-specialised with 2 and
    4 stages, persistent) takes the same bounded exit."""
    V, T = inputs.icosphere(3)
    n, k = T.shape[0], 1.0
    x = inputs.random_density(n, 1, seed=4, stream=0)
    y = inputs.random_density(n, 1, seed=4, stream=1)
    ref = oracle.apply(V, T, k, x=x, y=y)
    op = Operator(V, T, k, p=10, mode="mixed", leaf_level=3, tc_pipeline=pipeline)
    lib = _lib.load()
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()

    _lib.check(lib.bem_set_wait_limit(op._h, 1 << 14, 1))
    op.apply(xd, yd)  # stream-ordered: the expiry surfaces at the next synchronising call
    rc = lib.bem_sync(op._h, _stream())
    assert rc == _lib.BEM_ERR_TIMEOUT, rc
    assert b"bounded device wait" in lib.bem_last_error()

    # the flag is cleared when read, and the handle works normally again
    _lib.check(lib.bem_set_wait_limit(op._h, 0, 0))
    z = op.apply(xd, yd).cpu().numpy()
    _lib.check(lib.bem_sync(op._h, _stream()))
    err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    assert err <= 1e-5, err
    op.close()

