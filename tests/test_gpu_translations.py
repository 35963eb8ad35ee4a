"""Each stage of the far field against direct sums of the Green's function.

The FMM of Section 2.3 replaces far (target, source) pairs by expansions.
Here the expansions the library builds are read back (bem_far_field, in
textbook normalisation) and evaluated with scipy's spherical Bessel functions
and this file's own spherical harmonics, then compared with the direct sum of
the regular 3-point rule over the sources each expansion stands for:

  P2M, M2M  the multipole of every tree box, at points 3.5 box widths away,
            against the box's own elements (leaves: P2M alone; split boxes:
            M2M of their children);
  M2L, L2L, P2L  the local expansion of every tree box after the downward
            pass, at points inside the box, against every element whose box
            (on the local's level, or the element's leaf if that is coarser)
            does not touch it (level 2: M2L alone);
  L2P, M2P  the far-field part of z at every target, against every element
            whose leaf does not touch the target's leaf.

The meshes: a uniform tree on a sphere, and an adaptive tree split per box
(leaf_level = -2) on a unit sphere next to a finer sphere of radius 0.3, which
has leaves on several levels and therefore W- and X-lists (M2P, P2L).
"""
import ctypes

import numpy as np
import pytest
import torch
from scipy import special

from paper_1606_02383_gb300 import _lib, inputs
from paper_1606_02383_gb300.operator import Operator

pytestmark = pytest.mark.gpu


# ---------------------------------------------------------------- the test's own functions
def ylm(p, u):
    """Orthonormal Y_nm(u) without the Condon-Shortley phase, [K, (p+1)^2], index n^2+n+m."""
    ct = np.clip(u[:, 2], -1.0, 1.0)
    phi = np.arctan2(u[:, 1], u[:, 0])
    Y = np.zeros((u.shape[0], (p + 1) ** 2), dtype=np.complex128)
    for n in range(p + 1):
        for m in range(n + 1):
            lognorm = 0.5 * (np.log((2 * n + 1) / (4 * np.pi)) + special.gammaln(n - m + 1) - special.gammaln(n + m + 1))
            val = np.exp(lognorm) * special.lpmv(m, n, ct) * (-1.0) ** m * np.exp(1j * m * phi)
            Y[:, n * n + n + m] = val
            Y[:, n * n + n - m] = np.conj(val)
    return Y


def radial(p, x, outgoing):
    ns = np.arange(p + 1)
    j = special.spherical_jn(ns[None, :], x[:, None])
    if not outgoing:
        return j
    return j + 1j * special.spherical_yn(ns[None, :], x[:, None])


def eval_expansion(coef, p, k, centre, pts, outgoing):
    v = pts - centre[None, :]
    r = np.linalg.norm(v, axis=1)
    Y = ylm(p, v / r[:, None])
    R = radial(p, k * r, outgoing)
    nidx = np.floor(np.sqrt(np.arange((p + 1) ** 2))).astype(int)
    return (Y * R[:, nidx]) @ coef


def geometry(V, T):
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    cr = np.cross(b - a, c - a)
    area = 0.5 * np.linalg.norm(cr, axis=1)
    nrm = cr / (2.0 * area[:, None])
    w1, w2 = 2.0 / 3.0, 1.0 / 6.0
    q = np.stack([w1 * a + w2 * b + w2 * c, w2 * a + w1 * b + w2 * c, w2 * a + w2 * b + w1 * c], axis=1)
    return (a + b + c) / 3.0, area, nrm, q


def direct(pts, J, geo, k, x, y):
    """sum over elements J of the regular rule: (A/3) [G y - dG/dn_y x] at pts."""
    _, area, nrm, q = geo
    out = np.zeros(pts.shape[0], dtype=np.complex128)
    for s in range(3):
        d = q[J, s][None, :, :] - pts[:, None, :]           # y - x
        r = np.linalg.norm(d, axis=2)
        g = np.exp(1j * k * r) / (4 * np.pi * r)
        dg = g * (1j * k * r - 1.0) / r**2 * np.einsum("pjc,jc->pj", d, nrm[J])
        out += (g * y[J][None, :] - dg * x[J][None, :]) @ (area[J] / 3.0)
    return out


# ---------------------------------------------------------------- the library's tree and far field
class Tree:
    def __init__(self, op):
        lib = _lib.load()
        self.L = op.info("leaf_level")
        self.perm = np.empty(op.n, dtype=np.int32)
        _lib.check(lib.bem_sorted_order(op._h, self.perm.ctypes.data))
        self.levels = []
        for l in range(self.L + 1):
            nb = op.info(_lib.INFO_BOXES_OF_LEVEL + l)
            st, en = np.empty(nb, np.int32), np.empty(nb, np.int32)
            ce, fl = np.empty((nb, 3)), np.empty(nb, np.uint8)
            _lib.check(lib.bem_tree_level(op._h, l, st.ctypes.data, en.ctypes.data, ce.ctypes.data, fl.ctypes.data))
            self.levels.append((st, en, ce, fl))
        c0 = self.levels[0][2][0]
        self.w0 = 4.0 * np.abs(self.levels[1][2][0] - c0).max()
        # leaf of every element (caller order): level and box
        self.leaf_level = np.full(op.n, -1)
        self.leaf_box = np.full(op.n, -1)
        for l, (st, en, ce, fl) in enumerate(self.levels):
            for b in np.nonzero((fl & 1) & ~(fl >> 1) & 1)[0]:
                J = self.perm[st[b]:en[b]]
                self.leaf_level[J] = l
                self.leaf_box[J] = b
        assert (self.leaf_level >= 0).all()
        # box of every element on every level
        self.box_of = []
        for l, (st, en, ce, fl) in enumerate(self.levels):
            bo = np.empty(op.n, dtype=np.int64)
            for b in range(len(st)):
                bo[self.perm[st[b]:en[b]]] = b
            self.box_of.append(bo)

    def width(self, l):
        return self.w0 / 2.0 ** np.asarray(l)

    def touch(self, l1, c1, l2, c2):
        """Boxes (level l1, centre c1) and (l2, c2) touch or overlap (vectorised over rows)."""
        lim = 0.5 * (self.width(l1) + self.width(l2)) * (1 + 1e-9)
        return np.all(np.abs(np.atleast_2d(c1) - np.atleast_2d(c2)) <= np.atleast_1d(lim)[:, None], axis=1)

    def centres_at(self, lvl):
        """Centre of every element's box on level lvl[j] (rows)."""
        c = np.empty((len(lvl), 3))
        for l in np.unique(lvl):
            sel = lvl == l
            c[sel] = self.levels[l][2][self.box_of[l][sel]]
        return c


def far_field(op, x, y):
    lib = _lib.load()
    E = op.info("exp_total")
    M = torch.zeros((1, E), dtype=torch.complex128, device="cuda")
    L = torch.zeros_like(M)
    z = torch.zeros((1, op.n), dtype=torch.complex128, device="cuda")
    xd, yd = torch.from_numpy(x[None]).cuda(), torch.from_numpy(y[None]).cuda()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _lib.check(lib.bem_far_field(op._h, 1, _lib.BEM_C128, xd.data_ptr(), yd.data_ptr(), M.data_ptr(), L.data_ptr(),
                                 z.data_ptr(), s))
    return M.cpu().numpy()[0], L.cpu().numpy()[0], z.cpu().numpy()[0]


def two_spheres():
    V1, T1 = inputs.icosphere(3)
    V2, T2 = inputs.icosphere(3, 0.3, (1.3, 0.4, -0.2))
    return inputs.merge_meshes([(V1, T1), (V2, T2)])


# tolerances, in the max norm over each box's sample points: the FP32 paths'
# rounding (mixed: expansions summed with FP32 atomics over every V-, X-list
# and parent contribution, measured up to 1.1e-5) and the truncation left at
# the orders used (p = 16 on the uniform tree, 20 on the adaptive one, whose
# M2P and P2L converge more slowly than M2L between same-level boxes)
CASES = [("uniform sphere", "mixed", 3, 2e-5), ("uniform sphere", "fp64", 3, 5e-6),
         ("two spheres, split per box", "mixed", -2, 2e-5), ("two spheres, split per box", "fp64", -2, 5e-6)]


@pytest.mark.parametrize("name,mode,leaf,tol", CASES)
def test_far_field_stages_match_direct_sums(cuda_ok, name, mode, leaf, tol):
    V, T = inputs.icosphere(3) if name.startswith("uniform") else two_spheres()
    k, p = 2.0, (16 if leaf > 0 else 20)
    op = Operator(V, T, k, p=p, mode=mode, leaf_level=leaf, leaf_target=16 if leaf < 0 else 48, max_nrhs=1)
    n = T.shape[0]
    x = inputs.random_density(n, 1, seed=11, stream=0)[0]
    y = inputs.random_density(n, 1, seed=11, stream=1)[0]
    geo = geometry(V, T)
    tree = Tree(op)
    M, L, zfar = far_field(op, x, y)
    P = (p + 1) ** 2
    rng = np.random.default_rng(5)
    checked = {"p2m": 0, "m2m": 0, "local": 0}
    if leaf < 0:
        assert op.info("w_pairs") > 0 and op.info("x_pairs") > 0, "the adaptive case must exercise M2P and P2L"
        assert len({l for l in tree.leaf_level}) >= 2
    for l in range(2, tree.L + 1):
        st, en, ce, fl = tree.levels[l]
        base = op.info(_lib.INFO_EXP_BASE_OF_LEVEL + l)
        w = tree.width(l)
        boxes = np.nonzero(fl & 1)[0]
        for b in rng.choice(boxes, min(len(boxes), 24), replace=False):
            coef = slice(base + b * P, base + (b + 1) * P)
            # multipole: the box's own elements, seen from 3.5 widths away
            J = tree.perm[st[b]:en[b]]
            dirs = rng.standard_normal((6, 3))
            pts = ce[b] + 3.5 * w * dirs / np.linalg.norm(dirs, axis=1)[:, None]
            want = direct(pts, J, geo, k, x, y)
            got = eval_expansion(M[coef], p, k, ce[b], pts, outgoing=True)
            err = np.abs(got - want).max() / np.abs(want).max()
            assert err <= tol, ("multipole", name, mode, l, b, err)
            checked["m2m" if fl[b] & 2 else "p2m"] += 1
            # local: every element whose box on this level (or coarser leaf) does not touch b
            lvl_j = np.minimum(tree.leaf_level, l)
            far = ~tree.touch(lvl_j, tree.centres_at(lvl_j), np.full(n, l), ce[b][None, :])
            if not far.any():
                continue
            dirs = rng.uniform(-0.3, 0.3, size=(6, 3)) * w
            pts = ce[b] + dirs
            want = direct(pts, np.nonzero(far)[0], geo, k, x, y)
            got = eval_expansion(L[coef], p, k, ce[b], pts, outgoing=False)
            err = np.abs(got - want).max() / np.abs(want).max()
            assert err <= tol, ("local", name, mode, l, b, err)
            checked["local"] += 1
    assert checked["p2m"] > 0 and checked["local"] > 0
    # far part of z: every element whose leaf does not touch the target's leaf
    cen = geo[0]
    leaf_c = tree.centres_at(tree.leaf_level)
    for i in rng.choice(n, 40, replace=False):
        far = ~tree.touch(tree.leaf_level, leaf_c, np.full(n, tree.leaf_level[i]), leaf_c[i][None, :])
        want = direct(cen[i:i + 1], np.nonzero(far)[0], geo, k, x, y)[0]
        scale = np.abs(zfar).max()
        assert abs(zfar[i] - want) <= tol * scale, ("zfar", name, mode, i, abs(zfar[i] - want) / scale)
    op.close()
