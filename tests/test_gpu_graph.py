"""A setup-free apply is capturable into a CUDA graph and replays correctly.

The apply makes no host synchronisation, allocation or event call (with the
stage timers off), so torch.cuda.graph can capture one call and replay it on
new densities written into the captured input buffers.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1606_02383_gb300 import inputs
from paper_1606_02383_gb300.operator import Operator

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("mode,tol", [("direct64", 1e-10), ("mixed", 1e-5)])
def test_apply_replayed_from_cuda_graph(cuda_ok, mode, tol):
    V, T = inputs.icosphere(3)
    n, k = T.shape[0], 1.5
    op = Operator(V, T, k, p=10, mode=mode, leaf_level=0 if mode == "direct64" else 3, max_nrhs=2)
    x = torch.from_numpy(inputs.random_density(n, 2, seed=0, stream=0)).cuda()
    y = torch.from_numpy(inputs.random_density(n, 2, seed=0, stream=1)).cuda()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):
            op.apply(x, y)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        z = op.apply(x, y)
    for seed in (1, 2):
        xn = inputs.random_density(n, 2, seed=seed, stream=0)
        yn = inputs.random_density(n, 2, seed=seed, stream=1)
        x.copy_(torch.from_numpy(xn))
        y.copy_(torch.from_numpy(yn))
        graph.replay()
        torch.cuda.synchronize()
        zg = z.cpu().numpy()
        assert rel(zg, oracle.apply(V, T, k, x=xn, y=yn)) <= tol
        assert rel(zg, op.apply(x, y).cpu().numpy()) <= (1e-14 if mode == "direct64" else 1e-6)
    op.close()
