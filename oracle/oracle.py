"""ctypes front end of the FP64 CPU oracle (bem_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and bench.py's
CPU-baseline leg, never by the product library.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

FLAG_RULE1 = 1
FLAG_NO_REFINE = 2
FLAG_NO_HALF = 4

_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_i64 = ctypes.c_int64


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if _build.stale():
        path = _build.build()
    lib = ctypes.CDLL(path)
    lib.oracle_num_threads.restype = ctypes.c_int
    lib.oracle_geometry.argtypes = [_D, _i64, _I32, _i64, _D, _D, _D, _D]
    lib.oracle_entries.argtypes = [_D, _i64, _I32, _i64, ctypes.c_double, ctypes.c_int, _I64, _I64, _i64, _D]
    lib.oracle_apply.argtypes = [_D, _i64, _I32, _i64, ctypes.c_double, ctypes.c_int, ctypes.c_int, _D, _D, _D,
                                 _I64, _i64]
    lib.oracle_apply_adjoint.argtypes = [_D, _i64, _I32, _i64, ctypes.c_double, ctypes.c_int, ctypes.c_int, _D, _D, _D]
    lib.oracle_eval_points.argtypes = [_D, _i64, _I32, _i64, ctypes.c_double, ctypes.c_int, ctypes.c_int, _D, _D,
                                       _D, _i64, _D]
    lib.oracle_eval_points_grad.argtypes = [_D, _i64, _I32, _i64, ctypes.c_double, ctypes.c_int, ctypes.c_int, _D,
                                            _D, _D, _i64, _D]
    lib.oracle_assemble.argtypes = [_D, _i64, _I32, _i64, ctypes.c_double, ctypes.c_int, _D, _D]
    lib.oracle_lu_solve.argtypes = [_i64, _D, ctypes.c_int, _D]
    lib.oracle_grad.argtypes = [_D, _i64, _I32, _i64, ctypes.c_double, ctypes.c_int, ctypes.c_int, _D, _D, _D,
                                _I64, _i64, _D, _D]
    for f in (lib.oracle_geometry, lib.oracle_entries, lib.oracle_apply, lib.oracle_apply_adjoint,
              lib.oracle_eval_points, lib.oracle_eval_points_grad, lib.oracle_assemble, lib.oracle_lu_solve,
              lib.oracle_grad):
        f.restype = ctypes.c_int
    _lib = lib
    return lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(_D)


def _mesh(V, T):
    V = np.ascontiguousarray(V, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.int32)
    return V, T


def _cplx(a, nt):
    if a is None:
        return None, 0
    a = np.ascontiguousarray(np.atleast_2d(a), dtype=np.complex128)
    assert a.shape[1] == nt
    return a, a.shape[0]


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def geometry(V, T):
    """centroids [nt,3], areas [nt], unit normals [nt,3], longest edges [nt]."""
    V, T = _mesh(V, T)
    nt = T.shape[0]
    c = np.empty((nt, 3))
    a = np.empty(nt)
    n = np.empty((nt, 3))
    h = np.empty(nt)
    _load().oracle_geometry(_dp(V), V.shape[0], T.ctypes.data_as(_I32), nt, _dp(c), _dp(a), _dp(n), _dp(h))
    return c, a, n, h


def entries(V, T, k, ii, jj, flags=0):
    """(S_ij, D_ij) for index pairs."""
    V, T = _mesh(V, T)
    ii = np.ascontiguousarray(ii, dtype=np.int64)
    jj = np.ascontiguousarray(jj, dtype=np.int64)
    out = np.empty((ii.size, 2), dtype=np.complex128)
    _load().oracle_entries(_dp(V), V.shape[0], T.ctypes.data_as(_I32), T.shape[0], float(k), int(flags),
                           ii.ctypes.data_as(_I64), jj.ctypes.data_as(_I64), ii.size, out.ctypes.data_as(_D))
    return out[:, 0].copy(), out[:, 1].copy()


def apply(V, T, k, x=None, y=None, rows=None, flags=0):
    """z = (1/2 I - D) x + S y, [nrhs, nt] (or [nrhs, len(rows)])."""
    V, T = _mesh(V, T)
    nt = T.shape[0]
    xa, nx = _cplx(x, nt)
    ya, ny = _cplx(y, nt)
    nrhs = max(nx, ny)
    assert nrhs > 0 and (nx in (0, nrhs)) and (ny in (0, nrhs))
    if rows is not None:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        nrows = rows.size
    else:
        nrows = nt
    z = np.empty((nrhs, nrows), dtype=np.complex128)
    rc = _load().oracle_apply(_dp(V), V.shape[0], T.ctypes.data_as(_I32), nt, float(k), int(flags), nrhs,
                              _dp(xa), _dp(ya), z.ctypes.data_as(_D),
                              None if rows is None else rows.ctypes.data_as(_I64), nrows)
    assert rc == 0
    return z


def adjoint(V, T, k, g, flags=0):
    """(gx, gy) = ((1/2 I - D)^H g, S^H g)."""
    V, T = _mesh(V, T)
    nt = T.shape[0]
    ga, nrhs = _cplx(g, nt)
    gx = np.empty((nrhs, nt), dtype=np.complex128)
    gy = np.empty((nrhs, nt), dtype=np.complex128)
    rc = _load().oracle_apply_adjoint(_dp(V), V.shape[0], T.ctypes.data_as(_I32), nt, float(k), int(flags), nrhs,
                                      _dp(ga), gx.ctypes.data_as(_D), gy.ctypes.data_as(_D))
    assert rc == 0
    return gx, gy


def grad(V, T, k, g, x=None, y=None, vertices=None, flags=0):
    """Gradient of the real loss L with dL = sum Re(conj(g) dz), z = (1/2 I - D) x + S y.

    Returns (dV, dk): dV [nv, 3] and dk (float) for every vertex; with
    `vertices` given, dV [len(vertices), 3] for those vertices only (computed
    from the pairs that touch them) and dk None.  Forward-mode dual arithmetic
    over every rule-defined entry (bem_oracle_grad.c)."""
    V, T = _mesh(V, T)
    nt = T.shape[0]
    ga, ng = _cplx(g, nt)
    xa, nx = _cplx(x, nt)
    ya, ny = _cplx(y, nt)
    assert ng > 0 and nx in (0, ng) and ny in (0, ng)
    if vertices is None:
        dV = np.empty((V.shape[0], 3))
        dk = np.empty(1)
        sel, nsel = None, 0
    else:
        sel = np.ascontiguousarray(vertices, dtype=np.int64)
        nsel = sel.size
        dV = np.empty((nsel, 3))
        dk = None
    rc = _load().oracle_grad(_dp(V), V.shape[0], T.ctypes.data_as(_I32), nt, float(k), int(flags), ng, _dp(ga),
                             _dp(xa), _dp(ya), None if sel is None else sel.ctypes.data_as(_I64), nsel, _dp(dV),
                             _dp(dk))
    assert rc == 0
    return dV, (None if dk is None else float(dk[0]))


def eval_points(V, T, k, pts, x=None, y=None, flags=0):
    """sum_j S(p,j) y_j - D(p,j) x_j at off-surface points p."""
    V, T = _mesh(V, T)
    nt = T.shape[0]
    xa, nx = _cplx(x, nt)
    ya, ny = _cplx(y, nt)
    nrhs = max(nx, ny)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    out = np.empty((nrhs, pts.shape[0]), dtype=np.complex128)
    rc = _load().oracle_eval_points(_dp(V), V.shape[0], T.ctypes.data_as(_I32), nt, float(k), int(flags), nrhs,
                                    _dp(xa), _dp(ya), _dp(pts), pts.shape[0], out.ctypes.data_as(_D))
    assert rc == 0
    return out


def eval_points_grad(V, T, k, pts, x=None, y=None, flags=0):
    """grad_p of sum_j S(p,j) y_j - D(p,j) x_j at off-surface points, [nrhs, npts, 3]."""
    V, T = _mesh(V, T)
    nt = T.shape[0]
    xa, nx = _cplx(x, nt)
    ya, ny = _cplx(y, nt)
    nrhs = max(nx, ny)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    out = np.empty((nrhs, pts.shape[0], 3), dtype=np.complex128)
    rc = _load().oracle_eval_points_grad(_dp(V), V.shape[0], T.ctypes.data_as(_I32), nt, float(k), int(flags), nrhs,
                                         _dp(xa), _dp(ya), _dp(pts), pts.shape[0], out.ctypes.data_as(_D))
    assert rc == 0
    return out


def assemble(V, T, k, flags=0):
    """Dense (S, D), each complex [nt, nt]."""
    V, T = _mesh(V, T)
    nt = T.shape[0]
    S = np.empty((nt, nt), dtype=np.complex128)
    D = np.empty((nt, nt), dtype=np.complex128)
    rc = _load().oracle_assemble(_dp(V), V.shape[0], T.ctypes.data_as(_I32), nt, float(k), int(flags),
                                 S.ctypes.data_as(_D), D.ctypes.data_as(_D))
    assert rc == 0
    return S, D


def lu_solve(A, B):
    """Solve A X = B (B: [nrhs, n]) with the oracle's LU with partial pivoting."""
    A = np.array(A, dtype=np.complex128, order="C", copy=True)
    B = np.array(np.atleast_2d(B), dtype=np.complex128, order="C", copy=True)
    n = A.shape[0]
    rc = _load().oracle_lu_solve(n, A.ctypes.data_as(_D), B.shape[0], B.ctypes.data_as(_D))
    if rc != 0:
        raise np.linalg.LinAlgError("singular matrix")
    return B
