"""PyTorch-facing wrapper of the CUDA library.

torch supplies device memory and the current CUDA stream; every computation
happens inside libbem.so (see _lib.py).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _raw(t: torch.Tensor) -> torch.Tensor:
    """Contiguous memory holding the tensor's values: the library reads raw
    memory, so lazy conjugate / negative views are resolved first."""
    return t.resolve_conj().resolve_neg().contiguous()


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.complex128:
        return _lib.BEM_C128
    if t.dtype == torch.complex64:
        return _lib.BEM_C64
    raise TypeError("densities must be complex64 or complex128 tensors")


def _options(mode="mixed", leaf_level=0, leaf_target=48, max_nrhs=16, p_min=4, p_max=40, p_level=None, p2p_unit=64,
             tc_kslice=16, corr_rules32=0, tc_tf32=0, tc_pipeline=0, p2p_ctas=0, p2p_stage=0, grad_direct=0):
    levels = (ctypes.c_int * 11)(*([0] * 11))
    for lvl, order in (p_level or {}).items():
        levels[int(lvl)] = int(order)
    return _lib.BemOptions(ctypes.sizeof(_lib.BemOptions), _lib.MODES[mode], int(leaf_level), int(leaf_target),
                           int(max_nrhs), int(p_min), int(p_max), levels, int(p2p_unit), int(tc_kslice),
                           int(corr_rules32), int(tc_tf32), int(tc_pipeline), int(p2p_ctas), int(p2p_stage),
                           int(grad_direct))


class Operator:
    """z = (1/2 I - D) x + S y on a triangle mesh (see include/bem.h).

    Parameters: vertices [nv,3] float64, triangles [nt,3] int32 (host arrays),
    wavenumber k, order p (> 0 fixed, 0 = automatic from eps), eps, mode in
    {"mixed", "fp64", "direct64", "direct32"}, leaf_level (> 0 uniform tree
    with leaves on that level, 0 = uniform on the level the mesh's mean
    occupancy picks, -1 = adaptive with the depth chosen per level-2 region,
    -2 = adaptive split per box), leaf_target (mean elements per leaf the
    automatic and adaptive trees aim at), max_nrhs, p_level ({level: order} overrides),
    p2p_unit (most targets per near-field work unit: 16, 32, 64), tc_kslice
    (most 16-wide K stages per tensor-core translation job, 2..16),
    corr_rules32 (mixed modes: near-singular rules of non-self pairs in FP32),
    tc_tf32 (mixed mode: 3xTF32 translations instead of the FP16 split),
    tc_pipeline (mixed modes, the translation loop: 1 two-stage
    block-synchronous, 2 or 4 warp-specialised stages, 0 the default),
    p2p_ctas (FP32 FMM: > 0 runs the near field from this many resident CTAs
    per SM beside the far field, which starts first), p2p_stage (FP32 FMM:
    the near list's source elements staged in shared memory by cp.async),
    grad_direct (FMM modes: the vertex gradient's regular rule summed over all
    pairs instead of through the octree).
    """

    def __init__(self, vertices, triangles, k, p=0, eps=1e-5, mode="mixed", leaf_level=0, leaf_target=48,
                 max_nrhs=16, p_min=4, p_max=40, p_level=None, p2p_unit=64, tc_kslice=16, corr_rules32=0,
                 tc_tf32=0, tc_pipeline=0, p2p_ctas=0, p2p_stage=0, grad_direct=0):
        lib = _lib.load()
        V = np.ascontiguousarray(vertices, dtype=np.float64)
        T = np.ascontiguousarray(triangles, dtype=np.int32)
        mesh = _lib.BemMesh(V.shape[0], T.shape[0], V.ctypes.data, T.ctypes.data, 0)
        opt = _options(mode, leaf_level, leaf_target, max_nrhs, p_min, p_max, p_level, p2p_unit, tc_kslice,
                       corr_rules32, tc_tf32, tc_pipeline, p2p_ctas, p2p_stage, grad_direct)
        h = ctypes.c_void_p()
        _lib.check(lib.bem_setup(ctypes.byref(mesh), float(k), int(p), float(eps), ctypes.byref(opt), _stream(),
                                 ctypes.byref(h)))
        self._h = h
        self._lib = lib
        self.n = T.shape[0]
        self.vertices = V.copy()
        self.k = float(k)
        self.mode = mode
        self.max_nrhs = int(max_nrhs)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.bem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self, key):
        v = ctypes.c_int64()
        code = _lib.INFO[key] if isinstance(key, str) else int(key)
        _lib.check(self._lib.bem_info(self._h, code, ctypes.byref(v)))
        return int(v.value)

    def profile(self, enable=True):
        """Start (or stop) per-stage CUDA-event timing inside the library."""
        _lib.check(self._lib.bem_profile(self._h, 1 if enable else 0))

    def profile_read(self):
        """{stage: (milliseconds, launches)} summed since profile() was called."""
        n = len(_lib.STAGES)
        ms = (ctypes.c_double * n)()
        ln = (ctypes.c_int64 * n)()
        _lib.check(self._lib.bem_profile_read(self._h, ms, ln, n))
        return {st: (ms[i], int(ln[i])) for i, st in enumerate(_lib.STAGES)}

    def order_of_level(self, level):
        return self.info(_lib.INFO_ORDER_OF_LEVEL + int(level))

    def _prep(self, t, dtype):
        if t is None:
            return None
        t = torch.as_tensor(t)
        if t.dim() == 1:
            t = t[None, :]
        # the library reads raw memory: lazy conjugate / negative views are resolved
        return _raw(t.to(device="cuda", dtype=dtype))

    def apply(self, x=None, y=None, no_half=False, dtype=None):
        """z = (1/2 I - D) x + S y for device densities [nrhs, n] (or [n])."""
        ref = x if x is not None else y
        if ref is None:
            raise ValueError("x and y cannot both be None")
        dtype = dtype or (ref.dtype if isinstance(ref, torch.Tensor) else torch.complex128)
        xs, ys = self._prep(x, dtype), self._prep(y, dtype)
        nrhs = (xs if xs is not None else ys).shape[0]
        z = torch.empty((nrhs, self.n), dtype=dtype, device="cuda")
        flags = _lib.BEM_APPLY_NO_HALF if no_half else 0
        _lib.check(self._lib.bem_apply(self._h, nrhs, _dtype_code(z), None if xs is None else xs.data_ptr(),
                                       None if ys is None else ys.data_ptr(), z.data_ptr(), flags, _stream()))
        return z

    def eval_points(self, points, x=None, y=None, dtype=None, gradient=False, value_and_gradient=False,
                    direct=False):
        """u(p) = sum_j S(p, j) y_j - D(p, j) x_j at points [npoints, 3] off the
        surface.  Returns [nrhs, npoints]; grad u as [nrhs, npoints, 3] with
        gradient=True; (u, grad u) as [nrhs, npoints, 4] with
        value_and_gradient=True.  FMM handles walk the octree (multipoles of
        far boxes, rules on near leaves) unless direct=True asks for the
        direct sum over all elements."""
        ref = x if x is not None else y
        if ref is None:
            raise ValueError("x and y cannot both be None")
        if gradient and value_and_gradient:
            raise ValueError("gradient and value_and_gradient exclude each other")
        dtype = dtype or (ref.dtype if isinstance(ref, torch.Tensor) else torch.complex128)
        xs, ys = self._prep(x, dtype), self._prep(y, dtype)
        nrhs = (xs if xs is not None else ys).shape[0]
        pts = torch.as_tensor(points, dtype=torch.float64).reshape(-1, 3).to("cuda").contiguous()
        nc = 4 if value_and_gradient else (3 if gradient else 1)
        shape = (nrhs, pts.shape[0], nc) if nc > 1 else (nrhs, pts.shape[0])
        out = torch.empty(shape, dtype=dtype, device="cuda")
        flags = (_lib.BEM_EVAL_VALUE_GRADIENT if value_and_gradient else 0) | \
            (_lib.BEM_EVAL_GRADIENT if gradient else 0) | (_lib.BEM_EVAL_DIRECT if direct else 0)
        _lib.check(self._lib.bem_eval_points(self._h, nrhs, _dtype_code(out), None if xs is None else xs.data_ptr(),
                                             None if ys is None else ys.data_ptr(), pts.data_ptr(), pts.shape[0],
                                             out.data_ptr(), flags, _stream()))
        return out

    def point_sources(self, points, amps, dtype=torch.complex128):
        """b_i = sum_m a_m G(c_i - x_m) at the collocation points: points [nsrc, 3],
        amps [nrhs, nsrc] (or [nsrc]).  Returns [nrhs, N]."""
        pts = torch.as_tensor(points, dtype=torch.float64).reshape(-1, 3).to("cuda").contiguous()
        a = torch.as_tensor(amps).to("cuda", torch.complex128)
        a = _raw(a if a.dim() == 2 else a[None])
        if a.shape[1] != pts.shape[0]:
            raise ValueError("amps must be [nrhs, nsrc] with nsrc = len(points)")
        out = torch.empty((a.shape[0], self.n), dtype=dtype, device="cuda")
        _lib.check(self._lib.bem_point_sources(self._h, a.shape[0], _dtype_code(out), pts.shape[0], pts.data_ptr(),
                                               a.data_ptr(), out.data_ptr(), _stream()))
        return out

    def state_and_adjoint(self, b, observers, incident_at_observers, tol=1e-8, max_iter=200, restart=200,
                          driver="graph"):
        """The chain of Section 2.2 for f = 1/2 |p|^2 summed over observation points
        (one bem_state_adjoint call): the state solve (1/2 I - D) p = b; the
        pressure at the observers, p(x_m) = p_inc(x_m) + (D p)(x_m) (the rigid
        body's representation formula); the adjoint right-hand side
        sum_m conj(p(x_m)) G(c - x_m); the adjoint solve with the same
        operator.  Returns a dict with p, p_obs, weights, p_adj, iterations and
        residuals."""
        bs = self._prep(b, b.dtype)
        if bs.shape[0] != 1:
            raise ValueError("the chain takes one right-hand side")
        obs = torch.as_tensor(observers, dtype=torch.float64).reshape(-1, 3).to("cuda").contiguous()
        inc = _raw(torch.as_tensor(incident_at_observers).to("cuda", torch.complex128).reshape(-1))
        nobs = obs.shape[0]
        if inc.shape[0] != nobs:
            raise ValueError("one incident value per observer")
        p = torch.empty_like(bs)
        p_adj = torch.empty_like(bs)
        p_obs = torch.empty((1, nobs), dtype=torch.complex128, device="cuda")
        weights = torch.empty_like(p_obs)
        iters = (ctypes.c_int * 2)()
        rel = (ctypes.c_double * 2)()
        _lib.check(self._lib.bem_state_adjoint(self._h, _dtype_code(bs), bs.data_ptr(), nobs, obs.data_ptr(),
                                               inc.data_ptr(), float(tol), int(max_iter), int(restart),
                                               _gmres_driver_flags(driver), p.data_ptr(), p_obs.data_ptr(),
                                               weights.data_ptr(), p_adj.data_ptr(), iters, rel, _stream()))
        return {"p": p, "p_obs": p_obs, "weights": weights, "p_adj": p_adj, "iterations": (iters[0], iters[1]),
                "relres": (np.array([rel[0]]), np.array([rel[1]]))}

    def point_source_field(self, points, sources, amps, gradient=False):
        """phi(x) = sum_m a_m G(x - x_m) at points [npoints, 3] (with the
        gradient: [nrhs, npoints, 4] = phi, d/dx, d/dy, d/dz)."""
        pts = torch.as_tensor(points, dtype=torch.float64).reshape(-1, 3).to("cuda").contiguous()
        src = torch.as_tensor(sources, dtype=torch.float64).reshape(-1, 3).to("cuda").contiguous()
        a = torch.as_tensor(amps).to("cuda", torch.complex128)
        a = _raw(a if a.dim() == 2 else a[None])
        shape = (a.shape[0], pts.shape[0], 4) if gradient else (a.shape[0], pts.shape[0])
        out = torch.empty(shape, dtype=torch.complex128, device="cuda")
        _lib.check(self._lib.bem_point_source_field(a.shape[0], src.shape[0], src.data_ptr(), a.data_ptr(),
                                                    pts.shape[0], pts.data_ptr(), float(self.k),
                                                    _lib.BEM_EVAL_GRADIENT if gradient else 0, out.data_ptr(),
                                                    _stream()))
        return out

    def topological_derivative(self, points, chain, observers, incident, c1=1.5, c2=None):
        """T(x) = Re[c1 grad p . grad pa - c2 p pa] at points in the fluid
        (Section 2.5), from a state_and_adjoint result `chain` of the rigid
        body: p = p_inc + D p_surf and pa = phi + D pa_surf, phi the point
        sources at the observers with the adjoint weights (one
        bem_topological_field call).  incident: [npoints, 4] complex, the
        incident field and its gradient at the points (the caller's incident
        wave).  c1 = 3/2 and c2 = k^2 are the sound-hard limit in units
        rho_f = c_f = 1."""
        c2 = self.k ** 2 if c2 is None else float(c2)
        pts = torch.as_tensor(points, dtype=torch.float64).reshape(-1, 3).to("cuda").contiguous()
        inc = _raw(torch.as_tensor(incident).to("cuda", torch.complex128).reshape(-1, 4))
        obs = torch.as_tensor(observers, dtype=torch.float64).reshape(-1, 3).to("cuda").contiguous()
        w = _raw(torch.as_tensor(chain["weights"]).to("cuda", torch.complex128).reshape(-1))
        p = self._prep(chain["p"], chain["p"].dtype)
        pa = self._prep(chain["p_adj"], p.dtype)
        if inc.shape[0] != pts.shape[0] or w.shape[0] != obs.shape[0]:
            raise ValueError("incident must be [npoints, 4] and weights one per observer")
        T = torch.empty(pts.shape[0], dtype=torch.float64, device="cuda")
        _lib.check(self._lib.bem_topological_field(self._h, _dtype_code(p), p.data_ptr(), pa.data_ptr(), obs.shape[0],
                                                   obs.data_ptr(), w.data_ptr(), pts.shape[0], pts.data_ptr(),
                                                   inc.data_ptr(), float(c1), c2, T.data_ptr(), _stream()))
        return T

    def apply_host(self, x=None, y=None, out=None, no_half=False):
        """Same as apply() for host arrays/tensors (pinned is best); copies are inside the call."""
        x = None if x is None else _raw(x)
        y = None if y is None else _raw(y)
        ref = x if x is not None else y
        nrhs = ref.shape[0] if ref.dim() == 2 else 1
        dtype = ref.dtype
        if out is None:
            out = torch.empty((nrhs, self.n), dtype=dtype)
        flags = _lib.BEM_HOST_BUFFERS | (_lib.BEM_APPLY_NO_HALF if no_half else 0)
        _lib.check(self._lib.bem_apply(self._h, nrhs, _dtype_code(out), None if x is None else x.data_ptr(),
                                       None if y is None else y.data_ptr(), out.data_ptr(), flags, _stream()))
        return out

    def adjoint(self, g, no_half=False):
        """(gx, gy) = ((1/2 I - D)^H g, S^H g)."""
        gs = self._prep(g, g.dtype)
        nrhs = gs.shape[0]
        gx = torch.empty_like(gs)
        gy = torch.empty_like(gs)
        flags = _lib.BEM_APPLY_NO_HALF if no_half else 0
        _lib.check(self._lib.bem_apply_adjoint(self._h, nrhs, _dtype_code(gs), gs.data_ptr(), gx.data_ptr(),
                                               gy.data_ptr(), flags, _stream()))
        return gx, gy

    def grad_k(self, g, x=None, y=None):
        """dL/dk = sum Re <g, (dA/dk) u> for the upstream gradient g of z = apply(x, y)."""
        gs = self._prep(g, g.dtype)
        xs, ys = self._prep(x, g.dtype), self._prep(y, g.dtype)
        dk = ctypes.c_double(0.0)
        _lib.check(self._lib.bem_grad(self._h, gs.shape[0], _dtype_code(gs), gs.data_ptr(),
                                      None if xs is None else xs.data_ptr(), None if ys is None else ys.data_ptr(),
                                      None, ctypes.byref(dk), _stream()))
        return float(dk.value)

    def grad(self, g, x=None, y=None, vertices=True, k=True):
        """Gradients of the real loss with upstream gradient g of z = apply(x, y).

        Returns (dV, dk): dV a float64 array [nv, 3] of dL/dvertices (None when
        vertices=False) and dk = dL/dk (None when k=False), from one bem_grad call."""
        gs = self._prep(g, g.dtype)
        xs, ys = self._prep(x, g.dtype), self._prep(y, g.dtype)
        dV = np.zeros(self.vertices.shape, dtype=np.float64) if vertices else None
        dk = ctypes.c_double(0.0)
        _lib.check(self._lib.bem_grad(self._h, gs.shape[0], _dtype_code(gs), gs.data_ptr(),
                                      None if xs is None else xs.data_ptr(), None if ys is None else ys.data_ptr(),
                                      None if dV is None else dV.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      ctypes.byref(dk) if k else None,
                                      _stream()))
        return dV, (float(dk.value) if k else None)

    def __call__(self, x, y, k=None, vertices=None):
        """Differentiable z = (1/2 I - D) x + S y (torch.autograd).

        Backward: dL/dx, dL/dy from bem_apply_adjoint.  If a real tensor `k`
        (equal to the operator's wavenumber) or a float64 tensor `vertices`
        (equal to the mesh the operator was set up with) is passed, dL/dk and
        dL/dvertices come from bem_grad.
        """
        if k is None:
            k = torch.tensor(self.k, dtype=torch.float64)
        return BemApplyFn.apply(self, x, y, k, vertices)

    def solve(self, b, tol=1e-8, max_iter=200, restart=200, x0=None, raise_on_fail=True, driver="graph",
              coupling=None):
        """GMRES for (1/2 I - D) x = b.  Returns (x, iterations, relres[nrhs]).
        driver: "graph" (each restart cycle one CUDA graph, falling back to the
        host loop if no graph can be built), "graph_only" (no fallback) or
        "host" (the Arnoldi steps driven from the host).

        coupling: optional FemBody (the library's elastic body: the whole
        coupled solve runs in native code) or callable coupling(cx, cy) for
        Eq. (GMRES), (1/2 I - D + S C) x = b.  cx and cy are complex128 CUDA tensors
        [nrhs, N] at fixed addresses; the callable must write C cx into cy in
        place, on the current stream (e.g. the FEM map T (K - rho_s omega^2
        M)^{-1} N of Section 2.3).  A coupled solve runs the host loop."""
        bs = self._prep(b, b.dtype)
        nrhs = bs.shape[0]
        x = torch.zeros_like(bs) if x0 is None else self._prep(x0, bs.dtype).clone()
        iters = ctypes.c_int(0)
        rel = (ctypes.c_double * nrhs)()
        flags = (_lib.BEM_GMRES_USE_X0 if x0 is not None else 0) | _gmres_driver_flags(driver)
        if coupling is None:
            rc = self._lib.bem_gmres_solve(self._h, nrhs, _dtype_code(bs), bs.data_ptr(), x.data_ptr(), float(tol),
                                           int(max_iter), int(restart), flags, ctypes.byref(iters), rel, _stream())
        elif isinstance(coupling, FemBody):
            # the library's own coupling map: the whole solve stays in native code
            cx = torch.zeros((nrhs, self.n), dtype=torch.complex128, device="cuda")
            cy = torch.zeros_like(cx)
            _lib.check(self._lib.bem_fem_bind(coupling._f, cx.data_ptr(), cy.data_ptr()))
            fn = _lib.COUPLING_FN(ctypes.cast(self._lib.bem_fem_coupling, ctypes.c_void_p).value)
            rc = self._lib.bem_gmres_solve_coupled(self._h, nrhs, _dtype_code(bs), bs.data_ptr(), x.data_ptr(),
                                                   float(tol), int(max_iter), int(restart), fn, coupling._f,
                                                   cx.data_ptr(), cy.data_ptr(), flags, ctypes.byref(iters), rel,
                                                   _stream())
            self._lib.bem_fem_bind(coupling._f, None, None)
        else:
            cx = torch.zeros((nrhs, self.n), dtype=torch.complex128, device="cuda")
            cy = torch.zeros_like(cx)
            raised = []

            def _cb(_ctx, _nrhs, _stream_ptr):
                try:
                    coupling(cx, cy)
                    return 0
                except BaseException as e:  # an exception must not cross the C frames
                    raised.append(e)
                    return 1

            fn = _lib.COUPLING_FN(_cb)
            rc = self._lib.bem_gmres_solve_coupled(self._h, nrhs, _dtype_code(bs), bs.data_ptr(), x.data_ptr(),
                                                   float(tol), int(max_iter), int(restart), fn, None, cx.data_ptr(),
                                                   cy.data_ptr(), flags, ctypes.byref(iters), rel, _stream())
            if rc == _lib.BEM_ERR_CALLBACK and raised:
                raise raised[0]
        if rc != _lib.BEM_OK and (raise_on_fail or rc != _lib.BEM_ERR_NOT_CONVERGED):
            _lib.check(rc)
        return x, int(iters.value), np.array(list(rel))


class FemBody:
    """The elastic body of Section 2.3 on the GPU (see bem_fem_setup in
    include/bem.h): P1 tetrahedra, K - rho_s omega^2 M assembled and
    factorised once, and the coupling map C = rho_f omega^2 Avg
    (K - rho_s omega^2 M)^{-1} (-N) of Eq. (GMRES).  tris are the boundary
    faces (the BEM mesh, normals out of the body) over the same node array.
    Pass the body as Operator.solve(coupling=body)."""

    def __init__(self, nodes, tets, tris, lam, mu, rho_s, rho_f, omega, keep_matrix=False):
        lib = _lib.load()
        X = np.ascontiguousarray(nodes, dtype=np.float64)
        Tt = np.ascontiguousarray(tets, dtype=np.int32)
        Tr = np.ascontiguousarray(tris, dtype=np.int32)
        f = ctypes.c_void_p()
        _lib.check(lib.bem_fem_setup(X.ctypes.data, X.shape[0], Tt.ctypes.data, Tt.shape[0], Tr.ctypes.data,
                                     Tr.shape[0], float(lam), float(mu), float(rho_s), float(rho_f), float(omega),
                                     _lib.BEM_FEM_KEEP_MATRIX if keep_matrix else 0, _stream(), ctypes.byref(f)))
        self._f = f
        self._lib = lib
        self.n_dof = 3 * X.shape[0]
        self.n_tris = Tr.shape[0]

    def close(self):
        if getattr(self, "_f", None):
            self._lib.bem_fem_destroy(self._f)
            self._f = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self, key):
        v = ctypes.c_int64()
        _lib.check(self._lib.bem_fem_info(self._f, _lib.FEM_INFO[key], ctypes.byref(v)))
        return int(v.value)

    def solve(self, b):
        """(K - rho_s omega^2 M)^{-1} b for real b [m, n_dof] (or [n_dof])."""
        bb = torch.as_tensor(b, dtype=torch.float64).to("cuda").contiguous()
        one = bb.dim() == 1
        bb = bb.reshape(-1, self.n_dof)
        u = torch.empty_like(bb)
        _lib.check(self._lib.bem_fem_solve(self._f, bb.shape[0], bb.data_ptr(), u.data_ptr(), _stream()))
        return u[0] if one else u

    def couple(self, x):
        """C x for complex element pressures x [nrhs, n_tris] (or [n_tris])."""
        xx = torch.as_tensor(x).to("cuda")
        if not xx.is_complex():
            xx = xx.to(torch.complex128)
        xx = xx.contiguous()
        one = xx.dim() == 1
        xx = xx.reshape(-1, self.n_tris)
        y = torch.empty_like(xx)
        _lib.check(self._lib.bem_fem_couple(self._f, xx.shape[0], _dtype_code(xx), xx.data_ptr(), y.data_ptr(),
                                            _stream()))
        return y[0] if one else y

    def matrix(self):
        """The assembled K - rho_s omega^2 M (dense FP64, needs keep_matrix=True)."""
        out = torch.empty((self.n_dof, self.n_dof), dtype=torch.float64, device="cuda")
        _lib.check(self._lib.bem_fem_matrix(self._f, out.data_ptr(), _stream()))
        return out.T  # stored column-major


def isosurface(phi, lo, h, t=0.0):
    """The boundary {phi = t} of the level-set region {phi > t} (Section 2.4)
    as a closed triangle mesh, by marching tetrahedra on the CUDA device.

    phi: FP64 tensor [n0, n1, n2] (moved to the GPU), the value at
    lo + (i, j, k) h.  Returns (vertices [nv, 3] FP64, triangles [nt, 3] int32),
    CUDA tensors; triangles face out of {phi > t}, i.e. into the fluid."""
    lib = _lib.load()
    ph = phi.to(device="cuda", dtype=torch.float64).contiguous()
    if ph.dim() != 3:
        raise ValueError("phi must be [n0, n1, n2]")
    n0, n1, n2 = ph.shape
    lo3 = (ctypes.c_double * 3)(*[float(v) for v in lo])
    counts = (ctypes.c_int64 * 2)()
    _lib.check(lib.bem_isosurface(n0, n1, n2, ph.data_ptr(), lo3, float(h), float(t), None, 0, None, 0, counts,
                                  _stream()))
    V = torch.empty((max(int(counts[0]), 1), 3), dtype=torch.float64, device="cuda")
    T = torch.empty((max(int(counts[1]), 1), 3), dtype=torch.int32, device="cuda")
    _lib.check(lib.bem_isosurface(n0, n1, n2, ph.data_ptr(), lo3, float(h), float(t), V.data_ptr(), V.shape[0],
                                  T.data_ptr(), T.shape[0], counts, _stream()))
    return V[:int(counts[0])], T[:int(counts[1])]


def levelset_step(phi, t_omega, t_omegac, h, dt, C, tau, L, phi_bar, tol=1e-13, max_iter=10000,
                  raise_on_fail=True):
    """One step of the level-set update of Section 2.4 (see include/bem.h,
    bem_levelset_step) on CUDA float64 tensors of the lattice's shape.
    Returns (phi_new, iterations, relres)."""
    ph = torch.as_tensor(phi).to("cuda", torch.float64).contiguous()
    if ph.dim() != 3:
        raise ValueError("phi must be a 3-D lattice")
    ti = torch.as_tensor(t_omega).to("cuda", torch.float64).contiguous()
    to = torch.as_tensor(t_omegac).to("cuda", torch.float64).contiguous()
    if ti.shape != ph.shape or to.shape != ph.shape:
        raise ValueError("T_omega and T_omegac must have phi's shape")
    out = torch.empty_like(ph)
    lib = _lib.load()
    iters = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    n0, n1, n2 = ph.shape
    rc = lib.bem_levelset_step(n0, n1, n2, ph.data_ptr(), ti.data_ptr(), to.data_ptr(), float(h), float(dt), float(C),
                               float(tau), float(L), float(phi_bar), float(tol), int(max_iter), out.data_ptr(),
                               ctypes.byref(iters), ctypes.byref(rel), _stream())
    if rc != _lib.BEM_OK and (raise_on_fail or rc != _lib.BEM_ERR_NOT_CONVERGED):
        _lib.check(rc)
    return out, int(iters.value), float(rel.value)


def _gmres_driver_flags(driver):
    flags = {"graph": 0, "graph_only": _lib.BEM_GMRES_GRAPH_ONLY, "host": _lib.BEM_GMRES_HOST_LOOP}
    if driver not in flags:
        raise ValueError("driver must be 'graph', 'graph_only' or 'host'")
    return flags[driver]


class BemApplyFn(torch.autograd.Function):
    """z = (1/2 I - D) x + S y with the conjugate-transpose apply as its backward.

    For a linear map z = A u PyTorch's complex gradient convention gives
    grad_u = A^H grad_z, which is exactly bem_apply_adjoint.
    """

    @staticmethod
    def forward(ctx, op, x, y, k, vertices=None):
        if abs(float(k) - op.k) > 1e-12 * max(1.0, abs(op.k)):
            raise ValueError("k must equal the wavenumber the operator was set up with")
        if vertices is not None and not np.array_equal(vertices.detach().cpu().numpy(), op.vertices):
            raise ValueError("vertices must equal the mesh the operator was set up with")
        ctx.op = op
        ctx.save_for_backward(x, y)
        return op.apply(x, y)

    @staticmethod
    def backward(ctx, gz):
        x, y = ctx.saved_tensors
        gz = _raw(gz)
        gx, gy = ctx.op.adjoint(gz)
        gk = gv = None
        want_k, want_v = ctx.needs_input_grad[3], len(ctx.needs_input_grad) > 4 and ctx.needs_input_grad[4]
        if want_k or want_v:
            dV, dk = ctx.op.grad(gz, x, y, vertices=want_v, k=want_k)
            gk = torch.tensor(dk, dtype=torch.float64) if want_k else None
            gv = torch.from_numpy(dV) if want_v else None
        return None, gx.reshape(gz.shape), gy.reshape(gz.shape), gk, gv


class Batch:
    """Many independent problems (meshes with their own wavenumbers) applied together.

    problems: list of (vertices, triangles, k).  Densities are concatenated
    along the element axis in problem order: [nrhs, sum N_b].
    """

    def __init__(self, problems, p=0, eps=1e-5, mode="mixed", leaf_level=0, leaf_target=48, max_nrhs=4,
                 options=None):
        lib = _lib.load()
        self._keep = []
        meshes = (_lib.BemMesh * len(problems))()
        ks = (ctypes.c_double * len(problems))()
        for i, (V, T, k) in enumerate(problems):
            V = np.ascontiguousarray(V, dtype=np.float64)
            T = np.ascontiguousarray(T, dtype=np.int32)
            self._keep += [V, T]
            meshes[i] = _lib.BemMesh(V.shape[0], T.shape[0], V.ctypes.data, T.ctypes.data, 0)
            ks[i] = float(k)
        h = ctypes.c_void_p()
        if options is None:
            opt = _options(mode, leaf_level, leaf_target, max_nrhs)
            _lib.check(lib.bem_setup_batch(meshes, ks, len(problems), int(p), float(eps), ctypes.byref(opt),
                                           _stream(), ctypes.byref(h)))
        else:
            # per-problem options (e.g. an autotuner's choices): dicts of Operator keywords
            opts = (_lib.BemOptions * len(problems))()
            for i, o in enumerate(options):
                kw = {"mode": mode, "leaf_level": leaf_level, "leaf_target": leaf_target}
                kw.update(o or {})
                kw["max_nrhs"] = max_nrhs
                opts[i] = _options(**kw)
            _lib.check(lib.bem_setup_batch_each(meshes, ks, len(problems), int(p), float(eps), opts, _stream(),
                                                ctypes.byref(h)))
        self._h = h
        self._lib = lib
        self.sizes = [int(T.shape[0]) for _, T, _ in problems]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        self.n = int(self.offsets[-1])

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.bem_destroy_batch(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self, problem, key):
        v = ctypes.c_int64()
        code = _lib.INFO[key] if isinstance(key, str) else int(key)
        _lib.check(self._lib.bem_batch_info(self._h, int(problem), code, ctypes.byref(v)))
        return int(v.value)

    def apply(self, x=None, y=None, no_half=False):
        ref = x if x is not None else y
        dtype = ref.dtype
        xs = None if x is None else _raw((x if x.dim() == 2 else x[None]).to("cuda", dtype))
        ys = None if y is None else _raw((y if y.dim() == 2 else y[None]).to("cuda", dtype))
        nrhs = (xs if xs is not None else ys).shape[0]
        z = torch.empty((nrhs, self.n), dtype=dtype, device="cuda")
        _lib.check(self._lib.bem_apply_batch(self._h, nrhs, _dtype_code(z), None if xs is None else xs.data_ptr(),
                                             None if ys is None else ys.data_ptr(), z.data_ptr(),
                                             _lib.BEM_APPLY_NO_HALF if no_half else 0, _stream()))
        return z

    def solve(self, b, tol=1e-8, max_iter=200, restart=200, x0=None, raise_on_fail=True, driver="graph"):
        """GMRES for (1/2 I - D_p) x_p = b_p on every problem p at once (each with its
        own Krylov space).  b: [nrhs, N_total].  Returns (x, iterations,
        relres[nrhs, number of problems]).  driver as for Operator.solve."""
        bs = _raw((b if b.dim() == 2 else b[None]).to("cuda"))
        nrhs = bs.shape[0]
        x = torch.zeros_like(bs) if x0 is None else _raw((x0 if x0.dim() == 2 else x0[None]).to("cuda", bs.dtype)).clone()
        iters = ctypes.c_int(0)
        nprob = len(self.sizes)
        rel = (ctypes.c_double * (nrhs * nprob))()
        flags = (_lib.BEM_GMRES_USE_X0 if x0 is not None else 0) | _gmres_driver_flags(driver)
        rc = self._lib.bem_gmres_solve_batch(self._h, nrhs, _dtype_code(bs), bs.data_ptr(), x.data_ptr(), float(tol),
                                             int(max_iter), int(restart), flags, ctypes.byref(iters), rel, _stream())
        if rc != _lib.BEM_OK and (raise_on_fail or rc != _lib.BEM_ERR_NOT_CONVERGED):
            _lib.check(rc)
        return x, int(iters.value), np.array(list(rel)).reshape(nrhs, nprob)
