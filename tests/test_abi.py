"""The C ABI library loads and exports every entry point include/bem.h declares (no GPU needed)."""
import ctypes
import os
import re

from paper_1606_02383_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(?:int|const char\*)\s+(bem_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("bem_setup", "bem_destroy", "bem_apply", "bem_apply_adjoint", "bem_gmres_solve", "bem_info",
              "bem_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    build.build()
    lib = ctypes.CDLL(_lib.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(_lib.EXPORTS) <= set(_declared())


def test_error_paths_without_gpu():
    lib = _lib.load()
    h = ctypes.c_void_p()
    # NULL mesh -> invalid argument, no CUDA call needed
    rc = lib.bem_setup(None, 1.0, 8, 1e-5, None, None, ctypes.byref(h))
    assert rc == _lib.BEM_ERR_INVALID_ARG
    assert b"mesh" in lib.bem_last_error()
    mesh = _lib.BemMesh(3, 1, 0, 0, 0)
    assert lib.bem_setup(ctypes.byref(mesh), 1.0, 8, 1e-5, None, None, ctypes.byref(h)) == _lib.BEM_ERR_INVALID_ARG
    assert lib.bem_apply(None, 1, _lib.BEM_C128, None, None, None, 0, None) == _lib.BEM_ERR_INVALID_ARG
    assert lib.bem_destroy(None) == _lib.BEM_OK
    # the coupled solve checks its arguments before any CUDA call
    cb = _lib.COUPLING_FN(lambda ctx, nrhs, stream: 0)
    assert lib.bem_gmres_solve_coupled(None, 1, _lib.BEM_C128, None, None, 1e-8, 10, 10, cb, None, None, None, 0,
                                       None, None, None) == _lib.BEM_ERR_INVALID_ARG
    # the elastic body checks its arguments before any CUDA call
    out = ctypes.c_void_p()
    assert lib.bem_fem_setup(None, 8, None, 1, None, 1, 2.0, 1.0, 1.0, 1.0, 1.0, 0, None,
                             ctypes.byref(out)) == _lib.BEM_ERR_INVALID_ARG
    import numpy as _np
    X = _np.zeros((4, 3))
    tet = _np.array([[0, 1, 2, 4]], dtype=_np.int32)  # node 4 of 4: out of range
    tri = _np.array([[0, 1, 2]], dtype=_np.int32)
    assert lib.bem_fem_setup(X.ctypes.data, 4, tet.ctypes.data, 1, tri.ctypes.data, 1, 2.0, 1.0, 1.0, 1.0, 1.0, 0,
                             None, ctypes.byref(out)) == _lib.BEM_ERR_INVALID_ARG
    tet[0, 3] = 3
    assert lib.bem_fem_setup(X.ctypes.data, 4, tet.ctypes.data, 1, tri.ctypes.data, 1, 2.0, -1.0, 1.0, 1.0, 1.0, 0,
                             None, ctypes.byref(out)) == _lib.BEM_ERR_INVALID_ARG  # mu <= 0
    assert lib.bem_fem_solve(None, 1, None, None, None) == _lib.BEM_ERR_INVALID_ARG
    assert lib.bem_fem_couple(None, 1, _lib.BEM_C128, None, None, None) == _lib.BEM_ERR_INVALID_ARG
    assert lib.bem_fem_coupling(None, 1, None) == _lib.BEM_ERR_INVALID_ARG
    assert lib.bem_fem_matrix(None, None, None) == _lib.BEM_ERR_INVALID_ARG
    assert lib.bem_fem_destroy(None) == _lib.BEM_OK
    # the iso-surface checks its grid and level before any CUDA call
    lo = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    counts = (ctypes.c_int64 * 2)()
    fake = ctypes.c_void_p(16)  # never dereferenced: every case below fails its argument checks first
    assert lib.bem_isosurface(4, 4, 4, None, lo, 1.0, 0.0, None, 0, None, 0, counts, None) == _lib.BEM_ERR_INVALID_ARG
    assert lib.bem_isosurface(1, 4, 4, fake, lo, 1.0, 0.0, None, 0, None, 0, counts, None) == _lib.BEM_ERR_INVALID_ARG
    assert lib.bem_isosurface(4, 4, 4, fake, lo, 0.0, 0.0, None, 0, None, 0, counts, None) == _lib.BEM_ERR_INVALID_ARG
    assert lib.bem_isosurface(4, 4, 4, fake, lo, 1.0, float("nan"), None, 0, None, 0, counts,
                              None) == _lib.BEM_ERR_INVALID_ARG
    assert lib.bem_isosurface(2048, 2048, 2048, fake, lo, 1.0, 0.0, None, 0, None, 0, counts,
                              None) == _lib.BEM_ERR_INVALID_ARG
    assert b"32-bit" in lib.bem_last_error()


def test_lazy_conjugate_views_are_resolved_before_the_library_reads_memory():
    """torch.conj gives a view whose raw memory holds the unconjugated values;
    the binding must hand the library the conjugated numbers."""
    import torch
    from paper_1606_02383_gb300.operator import _raw
    a = torch.tensor([1 + 2j, 3 - 4j], dtype=torch.complex128)
    r = _raw(torch.conj(a))
    assert not r.is_conj()
    raw = torch.view_as_real(r).flatten().tolist()
    assert raw == [1.0, -2.0, 3.0, 4.0]
    r = _raw(-torch.conj(a))
    assert torch.view_as_real(r).flatten().tolist() == [-1.0, 2.0, -3.0, -4.0]


def test_sync_and_wait_limit_reject_null_handles():
    lib = _lib.load()
    assert lib.bem_sync(None, None) == _lib.BEM_ERR_INVALID_ARG
    assert lib.bem_set_wait_limit(None, 0, 0) == _lib.BEM_ERR_INVALID_ARG


def test_levelset_step_rejects_bad_arguments():
    lib = _lib.load()
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    assert lib.bem_levelset_step(0, 4, 4, None, None, None, 0.1, 0.1, 1.0, 1.0, 1.0, -0.5, 1e-10, 10, None,
                                 ctypes.byref(it), ctypes.byref(rel), None) == _lib.BEM_ERR_INVALID_ARG
    assert lib.bem_levelset_step(4, 4, 4, None, None, None, 0.1, 0.1, 1.0, 1.0, 1.0, -0.5, 1e-10, 10, None,
                                 ctypes.byref(it), ctypes.byref(rel), None) == _lib.BEM_ERR_INVALID_ARG


def test_chain_calls_reject_null_handles():
    lib = _lib.load()
    it = (ctypes.c_int * 2)()
    rel = (ctypes.c_double * 2)()
    assert lib.bem_state_adjoint(None, _lib.BEM_C128, None, 1, None, None, 1e-8, 10, 10, 0, None, None, None, None,
                                 it, rel, None) == _lib.BEM_ERR_INVALID_ARG
    assert lib.bem_topological_field(None, _lib.BEM_C128, None, None, 1, None, None, 1, None, None, 1.5, 1.0, None,
                                     None) == _lib.BEM_ERR_INVALID_ARG
    assert lib.bem_eval_points(None, 1, _lib.BEM_C128, None, None, None, 1, None,
                               _lib.BEM_EVAL_GRADIENT | _lib.BEM_EVAL_VALUE_GRADIENT, None) == _lib.BEM_ERR_INVALID_ARG


def test_option_checks_without_gpu():
    """Out-of-range tree and tile options are rejected before any device work."""
    import numpy as np
    lib = _lib.load()
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=np.float64)
    T = np.array([[0, 1, 2]], dtype=np.int32)
    mesh = _lib.BemMesh(3, 1, V.ctypes.data, T.ctypes.data, 0)
    h = ctypes.c_void_p()
    from paper_1606_02383_gb300.operator import _options
    for kw, word in (({"leaf_level": -3}, b"leaf_level"), ({"p2p_unit": 48}, b"p2p_unit"),
                     ({"tc_kslice": 1}, b"tc_kslice"), ({"tc_kslice": 17}, b"tc_kslice"),
                     ({"tc_pipeline": 5}, b"tc_pipeline")):
        opt = _options(**kw)
        rc = lib.bem_setup(ctypes.byref(mesh), 1.0, 8, 1e-5, ctypes.byref(opt), None, ctypes.byref(h))
        assert rc == _lib.BEM_ERR_INVALID_ARG, kw
        assert word in lib.bem_last_error(), (kw, lib.bem_last_error())
