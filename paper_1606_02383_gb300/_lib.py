"""ctypes binding of libbem.so (argument marshalling only).

Every step of the operator runs inside the CUDA library; this module only
passes pointers, sizes and the stream.  If the library is missing the import
fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libbem.so")

BEM_OK = 0
BEM_ERR_INVALID_ARG = 1
BEM_ERR_DEGENERATE_MESH = 2
BEM_ERR_CUDA = 3
BEM_ERR_OOM = 4
BEM_ERR_NOT_CONVERGED = 5
BEM_ERR_TIMEOUT = 6
BEM_ERR_NUMERIC = 7
BEM_ERR_UNSUPPORTED = 8
BEM_ERR_CALLBACK = 9

BEM_C64 = 1
BEM_C128 = 2

MODES = {"mixed": 0, "fp64": 1, "direct64": 2, "direct32": 3, "tf32": 4}

BEM_APPLY_NO_HALF = 1
BEM_HOST_BUFFERS = 2
BEM_GMRES_USE_X0 = 1
BEM_GMRES_HOST_LOOP = 2
BEM_GMRES_GRAPH_ONLY = 4
BEM_EVAL_GRADIENT = 1
BEM_EVAL_VALUE_GRADIENT = 2
BEM_EVAL_DIRECT = 4

INFO = {
    "n": 0, "leaf_level": 1, "n_leaves": 2, "p2p_pairs": 3, "corr_nnz": 4, "m2l_pairs": 5, "m2l_flops": 6,
    "p_leaf": 7, "p_top": 8, "mode": 9, "device_bytes": 10, "p2m_bytes": 11, "launches_last_apply": 12,
    "m2m_flops": 13, "l2l_flops": 14, "adaptive": 15, "row_coeffs": 16, "w_pairs": 17, "x_pairs": 18,
    "near_list": 19, "w_evals": 20, "x_evals": 21, "exp_total": 22, "tc_kind": 23,
}
STAGES = ("prologue", "p2p", "correction", "p2m", "m2m", "m2l", "l2l", "l2p", "epilogue")
FEM_INFO = {"dof": 0, "nodes": 1, "tets": 2, "tris": 3, "device_bytes": 4}
BEM_FEM_KEEP_MATRIX = 1
INFO_ORDER_OF_LEVEL = 100
INFO_LEAVES_OF_LEVEL = 200
INFO_BOXES_OF_LEVEL = 300
INFO_EXP_BASE_OF_LEVEL = 400

# every entry point declared in include/bem.h
EXPORTS = ("bem_setup", "bem_destroy", "bem_apply", "bem_apply_adjoint", "bem_gmres_solve", "bem_info",
           "bem_profile", "bem_profile_read", "bem_apply_noalloc", "bem_grad", "bem_setup_batch", "bem_apply_batch",
           "bem_batch_info", "bem_destroy_batch", "bem_gmres_solve_batch", "bem_last_error", "bem_peak_probe",
           "bem_eval_points", "bem_point_sources", "bem_point_source_field", "bem_topological_derivative",
           "bem_gmres_solve_coupled", "bem_isosurface", "bem_sync", "bem_set_wait_limit", "bem_tree_level", "bem_sorted_order", "bem_far_field",
           "bem_setup_batch_each", "bem_state_adjoint", "bem_topological_field", "bem_levelset_step",
           "bem_fem_setup", "bem_fem_destroy", "bem_fem_solve", "bem_fem_couple", "bem_fem_bind", "bem_fem_coupling",
           "bem_fem_matrix", "bem_fem_info")

# int (*bem_coupling_fn)(void* ctx, int nrhs, void* stream)
COUPLING_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p)


class BemMesh(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("n_triangles", ctypes.c_int64),
                ("vertices", ctypes.c_void_p), ("triangles", ctypes.c_void_p), ("on_device", ctypes.c_int)]


class BemOptions(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_int), ("mode", ctypes.c_int), ("leaf_level", ctypes.c_int),
                ("leaf_target", ctypes.c_int), ("max_nrhs", ctypes.c_int), ("p_min", ctypes.c_int),
                ("p_max", ctypes.c_int), ("p_level", ctypes.c_int * 11), ("p2p_unit", ctypes.c_int),
                ("tc_kslice", ctypes.c_int), ("corr_rules32", ctypes.c_int), ("tc_tf32", ctypes.c_int),
                ("tc_pipeline", ctypes.c_int), ("p2p_ctas", ctypes.c_int),
                ("p2p_stage", ctypes.c_int), ("grad_direct", ctypes.c_int)]


class BemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("bem error %d: %s" % (code, msg))
        self.code = code


_lib = None


def load(path: str | None = None):
    """Load libbem.so (raises if absent)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("CUDA library %s is missing: run __graft_entry__.build() (no CPU fallback exists)" % p)
    lib = ctypes.CDLL(p)
    vp, i, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    lib.bem_setup.argtypes = [ctypes.POINTER(BemMesh), ctypes.c_double, i, ctypes.c_double,
                              ctypes.POINTER(BemOptions), vp, ctypes.POINTER(vp)]
    lib.bem_destroy.argtypes = [vp]
    lib.bem_apply.argtypes = [vp, i, i, vp, vp, vp, i, vp]
    lib.bem_apply_adjoint.argtypes = [vp, i, i, vp, vp, vp, i, vp]
    lib.bem_apply_noalloc.argtypes = [vp, i, i, vp, vp, vp, i, vp]
    lib.bem_grad.argtypes = [vp, i, i, vp, vp, vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                             vp]
    lib.bem_gmres_solve.argtypes = [vp, i, i, vp, vp, ctypes.c_double, i, i, i, ctypes.POINTER(i),
                                    ctypes.POINTER(ctypes.c_double), vp]
    lib.bem_gmres_solve_coupled.argtypes = [vp, i, i, vp, vp, ctypes.c_double, i, i, COUPLING_FN, vp, vp, vp, i,
                                            ctypes.POINTER(i), ctypes.POINTER(ctypes.c_double), vp]
    lib.bem_isosurface.argtypes = [i, i, i, vp, ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.c_double, vp,
                                   i64, vp, i64, ctypes.POINTER(i64), vp]
    lib.bem_gmres_solve_batch.argtypes = [vp, i, i, vp, vp, ctypes.c_double, i, i, i, ctypes.POINTER(i),
                                          ctypes.POINTER(ctypes.c_double), vp]
    lib.bem_info.argtypes = [vp, i, ctypes.POINTER(i64)]
    lib.bem_profile.argtypes = [vp, i]
    lib.bem_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64), i]
    lib.bem_setup_batch.argtypes = [ctypes.POINTER(BemMesh), ctypes.POINTER(ctypes.c_double), i, i, ctypes.c_double,
                                    ctypes.POINTER(BemOptions), vp, ctypes.POINTER(vp)]
    lib.bem_setup_batch_each.argtypes = [ctypes.POINTER(BemMesh), ctypes.POINTER(ctypes.c_double), i, i,
                                         ctypes.c_double, vp, vp, ctypes.POINTER(vp)]
    lib.bem_apply_batch.argtypes = [vp, i, i, vp, vp, vp, i, vp]
    lib.bem_batch_info.argtypes = [vp, i, i, ctypes.POINTER(i64)]
    lib.bem_destroy_batch.argtypes = [vp]
    lib.bem_peak_probe.argtypes = [i, i, ctypes.POINTER(ctypes.c_double), vp]
    lib.bem_eval_points.argtypes = [vp, i, i, vp, vp, vp, i64, vp, i, vp]
    lib.bem_point_sources.argtypes = [vp, i, i, i, vp, vp, vp, vp]
    lib.bem_point_source_field.argtypes = [i, i, vp, vp, i64, vp, ctypes.c_double, i, vp, vp]
    lib.bem_topological_derivative.argtypes = [i64, ctypes.c_double, ctypes.c_double, vp, vp, vp, vp]
    lib.bem_sync.argtypes = [vp, vp]
    lib.bem_fem_setup.argtypes = [vp, i64, vp, i64, vp, i64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, i, vp, ctypes.POINTER(vp)]
    lib.bem_fem_destroy.argtypes = [vp]
    lib.bem_fem_solve.argtypes = [vp, i, vp, vp, vp]
    lib.bem_fem_couple.argtypes = [vp, i, i, vp, vp, vp]
    lib.bem_fem_bind.argtypes = [vp, vp, vp]
    lib.bem_fem_coupling.argtypes = [vp, i, vp]
    lib.bem_fem_matrix.argtypes = [vp, vp, vp]
    lib.bem_fem_info.argtypes = [vp, i, ctypes.POINTER(i64)]
    lib.bem_tree_level.argtypes = [vp, i, vp, vp, vp, vp]
    lib.bem_sorted_order.argtypes = [vp, vp]
    lib.bem_far_field.argtypes = [vp, i, i, vp, vp, vp, vp, vp, vp]
    lib.bem_set_wait_limit.argtypes = [vp, ctypes.c_longlong, i]
    lib.bem_state_adjoint.argtypes = [vp, i, vp, i, vp, vp, ctypes.c_double, i, i, i, vp, vp, vp, vp,
                                      ctypes.POINTER(i), ctypes.POINTER(ctypes.c_double), vp]
    lib.bem_topological_field.argtypes = [vp, i, vp, vp, i, vp, vp, i64, vp, vp, ctypes.c_double, ctypes.c_double,
                                          vp, vp]
    d = ctypes.c_double
    lib.bem_levelset_step.argtypes = [i, i, i, vp, vp, vp, d, d, d, d, d, d, d, i, vp, ctypes.POINTER(i),
                                      ctypes.POINTER(d), vp]
    lib.bem_last_error.restype = ctypes.c_char_p
    for f in ("bem_setup", "bem_destroy", "bem_apply", "bem_apply_adjoint", "bem_gmres_solve", "bem_info",
              "bem_profile", "bem_profile_read", "bem_apply_noalloc", "bem_grad", "bem_setup_batch",
              "bem_apply_batch", "bem_batch_info", "bem_destroy_batch", "bem_gmres_solve_batch", "bem_peak_probe",
              "bem_eval_points", "bem_point_sources", "bem_point_source_field", "bem_topological_derivative",
              "bem_gmres_solve_coupled", "bem_isosurface", "bem_sync", "bem_set_wait_limit", "bem_tree_level", "bem_sorted_order", "bem_far_field", "bem_setup_batch_each",
              "bem_state_adjoint", "bem_topological_field", "bem_levelset_step"):
        getattr(lib, f).restype = i
    _lib = lib
    return lib


def check(rc: int):
    if rc != BEM_OK:
        raise BemError(rc, load().bem_last_error().decode(errors="replace"))
