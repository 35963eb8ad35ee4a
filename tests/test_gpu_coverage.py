"""Every (target, source) pair is counted exactly once: near list, far field
or correction, never two of them and never none (the coverage requirement of
the FMM's interaction lists, Section 2.3).

The FMM is applied to the unit densities e_j for every element j, batched as
right-hand sides, and each result column is compared entry by entry with the
oracle's dense column.  A pair that the lists drop or count twice changes its
own entry by the whole entry, about 1e-2 of the column's norm on these meshes,
while at order p = 16 the FMM's truncation and FP32 rounding stay below
1e-5 of it (at p = 10 the double layer's worst entries, corner to corner
across one box, carry 1.5e-4 of truncation error, and both go to 1e-7 and
below as p grows in the FP64 mode: truncation, not coverage).  A
rel-L2 check of z = A x for random x would see the same mistake only as a
1/N-sized change.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1606_02383_gb300 import inputs
from paper_1606_02383_gb300.operator import Operator

pytestmark = pytest.mark.gpu

BATCH = 128


def _columns(op, n, which):
    """Columns of S (which = "S") or of -D (which = "D") through the apply."""
    out = np.empty((n, n), dtype=np.complex128)
    for j0 in range(0, n, BATCH):
        nb = min(BATCH, n - j0)
        e = torch.zeros((nb, n), dtype=torch.complex128, device="cuda")
        e[torch.arange(nb), torch.arange(j0, j0 + nb)] = 1.0
        z = op.apply(None, e) if which == "S" else op.apply(e, None, no_half=True)
        out[:, j0:j0 + nb] = z.cpu().numpy().T
    return out


def _check_columns(got, want, tol, label):
    colnorm = np.linalg.norm(want, axis=0)
    err = np.abs(got - want)
    rel_col = err / colnorm[None, :]
    worst = np.unravel_index(np.argmax(rel_col), rel_col.shape)
    assert rel_col.max() <= tol, "%s: entry (%d, %d) off by %.3e of its column's norm" % (
        label, worst[0], worst[1], rel_col.max())
    # a dropped or doubled pair is off by its whole entry: every entry that
    # matters (above 1e-2 of its column's norm) must be within 1e-2 of itself
    big = np.abs(want) >= 1e-2 * colnorm[None, :]
    rel_entry = np.where(big, err / np.where(big, np.abs(want), 1.0), 0.0)
    assert rel_entry.max() <= 1e-2, "%s: an entry is off by %.3e of itself" % (label, rel_entry.max())
    return float(rel_col.max())


@pytest.fixture(scope="module")
def sphere3_dense():
    V, T = inputs.icosphere(3)
    S, D = oracle.assemble(V, T, 1.0)
    return V, T, S, D


@pytest.mark.parametrize("mode,leaf", [("mixed", 2), ("mixed", 3), ("fp64", 2), ("fp64", 3)])
def test_every_pair_counted_once(cuda_ok, sphere3_dense, mode, leaf):
    V, T, S, D = sphere3_dense
    n = T.shape[0]
    op = Operator(V, T, 1.0, p=16, mode=mode, leaf_level=leaf, max_nrhs=BATCH)
    _check_columns(_columns(op, n, "S"), S, 1e-5, "%s leaf %d S" % (mode, leaf))
    _check_columns(_columns(op, n, "D"), -D, 1e-5, "%s leaf %d D" % (mode, leaf))
    op.close()


@pytest.mark.parametrize("mode,leaf,target", [("mixed", 2, 48), ("fp64", 2, 48), ("mixed", -2, 16), ("fp64", -2, 16),
                                              ("mixed", -1, 16)])
def test_every_pair_counted_once_two_bodies(cuda_ok, mode, leaf, target):
    """Two bodies of different size and element density in one tree: a unit
    sphere and a sphere of radius 0.3 at a distance, so that the boxes of the
    two differ in occupancy and in their neighbour structure.  With the
    adaptive trees (leaf_level -2: split per box, -1: depth per region) the
    leaves sit on several levels, so the near lists join leaves of different
    sizes and the W- and X-lists (M2P, P2L) carry part of the far field."""
    V1, T1 = inputs.icosphere(3 if leaf < 0 else 2)
    V2, T2 = inputs.icosphere(3 if leaf < 0 else 2, 0.3, (1.3, 0.4, -0.2))
    V, T = inputs.merge_meshes([(V1, T1), (V2, T2)])
    n = T.shape[0]
    S, D = oracle.assemble(V, T, 2.0)
    # p = 20 on the adaptive trees: their M2P and P2L converge more slowly
    op = Operator(V, T, 2.0, p=16 if leaf > 0 else 20, mode=mode, leaf_level=leaf, leaf_target=target,
                  max_nrhs=BATCH)
    if leaf == -2:
        assert op.info("w_pairs") > 0 and op.info("x_pairs") > 0
    if leaf < 0:
        levels = {l for l in range(11) if op.info(200 + l) > 0}
        assert len(levels) >= 2, levels
    label = "two bodies %s leaf %d" % (mode, leaf)
    _check_columns(_columns(op, n, "S"), S, 1e-5, label + " S")
    _check_columns(_columns(op, n, "D"), -D, 1e-5, label + " D")
    op.close()
