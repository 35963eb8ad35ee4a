/*
 * bem.h -- C ABI of the GB300 fast multipole BEM operator library.
 *
 * The library applies the discretised 3-D Helmholtz boundary operators of the
 * acoustic boundary integral equation (paper: Section 2.3, Eq. (danseibie2);
 * block system Eq. (renritupu); FMM step 2(c) of the solver algorithm):
 *
 *     z = (1/2 I - D) x + S y
 *
 * for flat triangles Gamma_j with piecewise-constant densities, collocation at
 * the triangle centroids x_i, G(r) = exp(i k r)/(4 pi r), and n_j the unit
 * normal pointing out of the scatterer into the fluid (Section 2.1).  The
 * paper fixes no quadrature, so matrix entries are defined by this rule: the
 * 3-point rule with barycentric points (2/3,1/6,1/6) and permutations; the
 * triangle split uniformly L times near the target (L = 2 when the target is
 * within 2 h_j of the centroid c_j, L = 1 within 4 h_j, h_j the longest edge);
 * and the exact integral for the self term (D_ii = 0 on a flat element).
 * The far field is evaluated by a fast multipole method on an octree
 * (Section 2.3, "a low-frequency FMM is employed"; truncation chosen so the
 * error is below the requested tolerance, Section 3).
 *
 * Conventions for every entry point:
 *  - Return value: a bem_status code; bem_last_error() gives a message
 *    (thread-local, valid until the next call on the same thread).
 *  - Device arrays are raw CUDA device pointers; complex arrays are
 *    interleaved (re, im) of the given bem_dtype, layout [nrhs][n] with the
 *    element index fastest, in the caller's triangle order.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Apply calls are stream-ordered and do not synchronise the
 *    host unless BEM_HOST_BUFFERS is given.
 *  - The caller owns every buffer it passes; the handle owns all device state
 *    it allocates at setup (geometry, tree, lists, translation operators,
 *    correction matrix, workspaces).
 *  - A handle must not be used from two host threads or two streams at once.
 *  - Nothing traps or exits on the device; device-detected problems are
 *    reported through the status of the next synchronising call.
 */
#ifndef BEM_H_
#define BEM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bem_handle bem_handle;

typedef enum {
  BEM_OK = 0,
  BEM_ERR_INVALID_ARG = 1,     /* null pointer, bad size, k <= 0, bad flags */
  BEM_ERR_DEGENERATE_MESH = 2, /* zero-area or non-finite triangle */
  BEM_ERR_CUDA = 3,            /* a CUDA runtime call failed */
  BEM_ERR_OOM = 4,             /* device allocation failed */
  BEM_ERR_NOT_CONVERGED = 5,   /* GMRES hit max_iter; x holds the last iterate */
  BEM_ERR_TIMEOUT = 6,         /* a bounded device wait expired */
  BEM_ERR_NUMERIC = 7,         /* NaN/Inf detected, or an unusable expansion */
  BEM_ERR_UNSUPPORTED = 8,     /* option combination not available */
  BEM_ERR_CALLBACK = 9         /* a caller's callback returned non-zero */
} bem_status;

typedef enum { BEM_C64 = 1, BEM_C128 = 2 } bem_dtype;

/* How the operator is evaluated (fixed at setup). */
typedef enum {
  BEM_MODE_FMM_MIXED = 0,   /* FP32 near field and expansions, FP64 setup, FP64 accumulation */
  BEM_MODE_FMM_FP64 = 1,    /* every stage in FP64 */
  BEM_MODE_DIRECT_FP64 = 2, /* O(N^2) direct sum in FP64 (same rule-defined operator) */
  BEM_MODE_DIRECT_FP32 = 3, /* O(N^2) direct sum in FP32 with FP64 correction */
  BEM_MODE_FMM_TF32 = 4     /* diagnostic: as MIXED but the translations use one plain TF32
                               product instead of the 3xTF32 split (shows what the split buys) */
} bem_mode;

/* bem_apply flags */
#define BEM_APPLY_NO_HALF 1     /* omit the 1/2 I term: z = -D x + S y */
#define BEM_HOST_BUFFERS 2      /* x, y, z are host pointers (pinned is best); the call
                                   copies in, computes, copies out and synchronises */

typedef struct {
  int64_t n_vertices;
  int64_t n_triangles;
  const double* vertices;    /* [n_vertices][3] */
  const int32_t* triangles;  /* [n_triangles][3], ordered so that (b-a)x(c-a) points
                                out of the scatterer into the fluid */
  int on_device;             /* 0: host pointers, 1: device pointers */
} bem_mesh;

typedef struct {
  int struct_size;  /* sizeof(bem_options); 0 means "all defaults" */
  int mode;         /* bem_mode, default BEM_MODE_FMM_MIXED */
  int leaf_level;   /* octree leaves (Section 2.3's FMM tree):
                       > 0  : uniform tree, every leaf on this level;
                       0    : uniform tree on the deepest level whose mean
                              occupancy over the mesh reaches leaf_target and
                              whose boxes are at least 3 longest edges wide
                              (the default);
                       -1   : adaptive, depth chosen per level-2 region: the
                              deepest level whose mean occupancy in the region
                              reaches leaf_target and whose boxes stay at least
                              3 of the region's longest edges wide;
                       -2   : adaptive, every box split while it holds more than
                              2 leaf_target elements and its children stay at
                              least 3 of its longest edges wide */
  int leaf_target;  /* mean triangles per occupied leaf for the automatic choice (default 48) */
  int max_nrhs;     /* largest nrhs a later call may use (default 16) */
  int p_min;        /* lower bound of the automatic per-level order (default 4) */
  int p_max;        /* upper bound of any order (default 40) */
  int p_level[11];  /* > 0: expansion order of octree level l (overrides p and eps there);
                       this is what the order autotuner sets */
  int p2p_unit;     /* most targets per near-field warp work unit: 16, 32 or 64 (default 64) */
  int tc_kslice;    /* most 16-wide K stages per tensor-core translation job, 2..16 (default 16) */
  int corr_rules32; /* mixed modes: 1 sums the refined rules of non-self near-singular pairs in FP32
                       relative to the target (faster setup); 0 sums them in FP64 (default) */
  int tc_tf32;      /* mixed mode: 1 runs the tensor-core translations as 3xTF32; 0 (default) as the
                       two-term FP16 split with power-of-two row scales (same 11-bit mantissa, half
                       the bytes and twice the tensor rate) */
  int tc_pipeline;  /* mixed modes, the tensor-core translation loop: 1 two stages, all threads gather,
                       synchronise, one thread issues the MMAs; 2 or 4 stages with specialised warps
                       (cp.async gather warps, a bulk-copy thread and an MMA thread, synchronised by
                       mbarriers alone; 2 stages leave room for two CTAs per SM); 3 persistent, one CTA
                       per SM walking the job list on a 3-stage ring with two tensor-memory accumulators
                       (the epilogue of one job overlaps the next); 0 (default) per operator: 3 for
                       M2M (few long jobs), 2 for M2L and L2L */
  int p2p_ctas;     /* FP32 FMM: > 0 forks the far field before the near field and runs the near field
                       from this many resident CTAs per SM (a work queue over its units), so that the
                       far field's kernels share the SMs with it; 0 (default) runs the near field on
                       the whole grid first and the far field after it */
  int p2p_stage;    /* FP32 FMM: 1 stages the near list's source elements in shared memory (per warp,
                       two buffers of 32 elements filled by cp.async while the other is summed);
                       0 (default) loads them from global memory in the loop */
  int grad_direct;  /* FMM modes: 1 sums the regular-rule part of the vertex gradient (bem_grad) directly
                       over all pairs, O(N^2); 0 (default) through the octree: the target side by the
                       walk of bem_eval_points at the centroids, the source side by a walk at the
                       quadrature points over the multipoles of point charges at the centroids */
} bem_options;

/*
 * bem_setup -- build everything that does not depend on the densities.
 *   mesh   : surface mesh, copied at setup (host or device pointers).
 *   k      : wavenumber k_f > 0 (Section 2.1, Eq. (kf)).
 *   p      : > 0 fixes the expansion order on every level; <= 0 picks the
 *            order of each level from eps (Section 3: truncation error < tol).
 *   eps    : target relative truncation error for the automatic order.
 *   opt    : nullable, see bem_options.
 *   stream : stream for the setup work; setup synchronises it before returning.
 *   out    : receives the new handle (NULL on failure).
 * Errors: INVALID_ARG, DEGENERATE_MESH, CUDA, OOM, NUMERIC.
 */
int bem_setup(const bem_mesh* mesh, double k, int p, double eps, const bem_options* opt, void* stream,
              bem_handle** out);

/* bem_destroy -- free a handle and all its device memory (NULL is accepted). */
int bem_destroy(bem_handle* h);

/*
 * bem_apply -- z = (1/2 I - D) x + S y  (Section 2.3, step 2(c)).
 *   nrhs  : number of right-hand sides, 1 <= nrhs <= max_nrhs.
 *   dtype : BEM_C64 or BEM_C128 for x, y and z.
 *   x     : D-density [nrhs][N], nullable (treated as zero).
 *   y     : S-density [nrhs][N], nullable (treated as zero).
 *   z     : output [nrhs][N]; must not alias x or y.
 *   flags : BEM_APPLY_NO_HALF, BEM_HOST_BUFFERS.
 */
int bem_apply(bem_handle* h, int nrhs, int dtype, const void* x, const void* y, void* z, int flags, void* stream);

/*
 * bem_apply_noalloc -- bem_apply for callers that cannot allocate device
 * memory.  (No counterpart in the paper: this is an interface convenience.)
 *
 * Who needs it: programs whose device memory belongs to an allocator or pool
 * that already holds the whole GPU, so a cudaMalloc would fail or fragment the
 * pool, and latency-critical loops that must stay out of the driver's
 * allocation path (cudaMalloc/cudaFree may synchronise the device).
 *
 * It computes exactly what bem_apply computes, with the same arguments, on
 * device buffers only (flags: BEM_APPLY_NO_HALF; BEM_HOST_BUFFERS is
 * rejected).  The per-call scratch (weighted densities, near/far partial sums,
 * expansions) lives in one fixed library array of BEM_NOALLOC_SCRATCH_BYTES
 * on each device instead of the handle's workspaces, and the call makes no
 * cudaMalloc, cudaFree or other allocating call.  The caller still passes x, y
 * and z; the handle comes from bem_setup, which did allocate.
 *  - nrhs is limited to [1, max_nrhs] as for bem_apply.
 *  - Limit: the scratch needed is the sum of four areas, each rounded up to
 *    256 bytes: densities nrhs * 16 N (mixed modes) or nrhs * 32 N (FP64
 *    modes), near and far sums 2 * nrhs * 16 N, and multipole plus local
 *    expansions 2 * nrhs * 8 E (mixed) or 2 * nrhs * 16 E (FP64), with E the
 *    number of expansion coefficients of the tree: about nrhs * (48 N + 16 E)
 *    bytes in the mixed modes and nrhs * (64 N + 32 E) in the FP64 modes.  A
 *    call that needs more than the array returns BEM_ERR_INVALID_ARG with the
 *    byte counts in bem_last_error().  At N = 327,680 (mixed) one call fits
 *    two right-hand sides.
 *  - While the call runs, the handle's workspace pointers point into the
 *    array; no other thread may use the same handle (bem_apply,
 *    bem_apply_adjoint, bem_eval_points, ...) until the call returns.
 *  - Every GPU that loads the library holds the array until the process exits.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current) and caches it; make that
 *    first call before any stream capture.
 *  - All calls share the array and it keeps the last call's contents: the
 *    call zeroes what must start at zero itself, and calls that overlap on the
 *    GPU (two streams, two threads, two handles) race on it.
 */
#define BEM_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
int bem_apply_noalloc(bem_handle* h, int nrhs, int dtype, const void* x, const void* y, void* z, int flags,
                      void* stream);

/*
 * bem_apply_adjoint -- conjugate transpose of bem_apply:
 *   gx = (1/2 I - D)^H g,  gy = S^H g   (either output nullable, not both).
 * The adjoint problem of Section 2.2 uses the same operator; this entry point
 * is what reverse-mode differentiation of bem_apply needs (PyTorch's complex
 * convention: the gradient of a linear map A is A^H applied to the output
 * gradient).  Every part of the apply is transposed exactly (near field,
 * correction, each FMM translation), so <A x, g> = <x, A^H g> holds to
 * rounding, not only to the FMM tolerance.
 *   g     : [nrhs][N] device buffer; gx, gy: [nrhs][N] device buffers.
 *   flags : BEM_APPLY_NO_HALF (gx = -D^H g).  Host buffers are not accepted.
 * The first call builds the transposed translation operators (allocation,
 * synchronising); later calls are stream-ordered like bem_apply.
 */
int bem_apply_adjoint(bem_handle* h, int nrhs, int dtype, const void* g, void* gx, void* gy, int flags,
                      void* stream);

/*
 * bem_grad -- derivatives of a real loss L with respect to the vertex
 * positions and the wavenumber k, given the upstream gradient g = dL/dz of
 * z = bem_apply(x, y) (PyTorch's convention for complex outputs:
 * g = dL/dRe z + i dL/dIm z), so that dL = sum over rhs of Re <g, dz>:
 *     dvertices[v] = sum over rhs of Re < g, (dA/dV_v) u >,
 *     dk           = sum over rhs of Re < g, (dA/dk) u >,
 * where A u = (1/2 I - D) x + S y and every rule-defined entry is
 * differentiated: the collocation point (the centroid) and the quadrature
 * points move with the vertices, the weight with the area and D with the unit
 * normal; the refined near-singular rules are differentiated point by point
 * (their refinement level is piecewise constant); the exact self term S_ii
 * in closed radial form (D_ii = 0 for every vertex position).  The k-kernels
 * are dG/dk = i exp(ikr)/(4 pi) and d(dG/dn)/dk = -k exp(ikr) (y-x).n/(4 pi r).
 * The gradients with respect to x and y are bem_apply_adjoint.
 *   g, x, y   : [nrhs][N] device buffers (x or y may be NULL, not both).
 *   dvertices : nullable host array [nv][3], the caller's vertex order
 *               (BEM_ERR_INVALID_ARG for a device pointer).
 *   dk        : nullable host pointer to one double; not both NULL.
 * Cost: direct sums over all pairs (O(N^2)): FP64 in the FP64 modes; in the
 * mixed modes FP32 with FP64 accumulation, and FP64 for pairs within 4.5
 * longest edges.  The correction pairs are FP64.  The call allocates per-call scratch and synchronises
 * `stream`.
 */
int bem_grad(bem_handle* h, int nrhs, int dtype, const void* g, const void* x, const void* y, double* dvertices,
             double* dk, void* stream);

/*
 * bem_eval_points -- the field of the densities at points off the surface:
 *   u(p) = sum_j S(p, j) y_j - D(p, j) x_j
 * (the representation formula's layer potentials, Section 2.1, at field
 * points instead of collocation points; the same rule-defined entries: R_2
 * within 2 h_j of element j's centroid, R_1 within 4 h_j, R_0 beyond; no
 * free term and no self term).
 *   x, y     : densities [nrhs][N] (device, dtype), either may be NULL.
 *   points   : [npoints][3] FP64 coordinates (device), anywhere off the
 *              surface (inside or outside the tree's root cube).
 *   out      : [nrhs][npoints][ncomp] complex (device, dtype): ncomp = 1, u(p)
 *              (flags 0); 3, grad u(p) (BEM_EVAL_GRADIENT); 4, u(p) and
 *              grad u(p) (BEM_EVAL_VALUE_GRADIENT).  The gradient is with
 *              respect to the field point (the same rules applied to grad G
 *              and grad dG/dn_y).
 *   flags    : at most one of BEM_EVAL_GRADIENT, BEM_EVAL_VALUE_GRADIENT;
 *              BEM_EVAL_DIRECT takes the direct sum on an FMM handle.
 * Cost, FMM handles (the default there): the upward pass (P2M, M2M) of the
 * densities, then for every point a walk of the octree from level 2: a box
 * that does not touch the point's box on its own level, and lies at least
 * 4 h_max(box) from the point's finest-level box, is taken through its
 * multipole (M2P, the handle's orders); a leaf that does is summed element by
 * element with the rules above; other boxes are opened.  About
 * O(npoints (189 P log N + near elements)).  Allocates its temporaries
 * (sorted points, FP64 partial sums: 16 ncomp nrhs npoints bytes and 36
 * npoints more) stream-ordered and frees them before it returns.
 * Cost, direct handles or BEM_EVAL_DIRECT: a direct sum over all elements for
 * every point (O(npoints N)); each block of 128 consecutive points shares one
 * FP32 origin, so consecutive points should be close to each other (a lattice
 * in its natural order).  No allocation.
 * Precision: the handle's (FP32 sums with FP64 between tiles and stages in
 * the mixed modes, FP64 in the FP64 modes); pairs within 4 h_j take the
 * refined rule from the FP64 geometry.  Stream-ordered; no host
 * synchronisation.
 */
#define BEM_EVAL_GRADIENT 1
#define BEM_EVAL_VALUE_GRADIENT 2
#define BEM_EVAL_DIRECT 4
int bem_eval_points(bem_handle* h, int nrhs, int dtype, const void* x, const void* y, const double* points,
                    int64_t npoints, void* out, int flags, void* stream);

/*
 * bem_point_sources -- b_i = sum_m a_m G(c_i - x_m), G = exp(ikr)/(4 pi r), at
 * the collocation points c_i (the adjoint right-hand side of Section 2.2:
 * point sources at the observation points x_m with weights a_m).
 *   points : [nsrc][3] FP64 (device), off the surface.
 *   amps   : [nrhs][nsrc] complex128 (device).
 *   out    : [nrhs][N] complex of dtype (device), caller's element order.
 * FP64, one thread per element.  Stream-ordered.
 */
int bem_point_sources(bem_handle* h, int nrhs, int dtype, int nsrc, const double* points, const double* amps,
                      void* out, void* stream);

/*
 * bem_point_source_field -- phi(x) = sum_m a_m G(x - x_m) (and grad phi) at
 * arbitrary points: the incident field of the adjoint problem of Section 2.2
 * (point sources at the observation points) anywhere in the fluid.
 *   src    : [nsrc][3] FP64 (device);  amps : [nrhs][nsrc] complex128 (device).
 *   points : [npoints][3] FP64 (device), away from the sources.
 *   flags  : 0, or BEM_EVAL_GRADIENT for (phi, d/dx, d/dy, d/dz) per point.
 *   out    : complex128 [nrhs][npoints] or [nrhs][npoints][4] (device).
 * FP64, one thread per point; no handle needed.  Stream-ordered.
 */
int bem_point_source_field(int nrhs, int nsrc, const double* src, const double* amps, int64_t npoints,
                           const double* points, double k, int flags, double* out, void* stream);

/*
 * bem_topological_derivative -- T(x) = Re[c1 grad p . grad pa - c2 p pa] at
 * points x from the state field p and the adjoint field pa (Section 2.5, the
 * topological derivative for an elastic inclusion appearing in the fluid:
 * c1 = 3 (rho_s - rho_f)/(2 rho_s + rho_f), c2 = rho_f omega^2
 * (Lambda_s - Lambda_f)/(Lambda_s Lambda_f); sound-hard limit c1 = 3/2).
 *   state, adjoint : complex128 [npoints][4] (device): the field and its three
 *                    gradient components at every point.
 *   T              : FP64 [npoints] (device).
 */
int bem_topological_derivative(int64_t npoints, double c1, double c2, const double* state, const double* adjoint,
                               double* T, void* stream);

/*
 * bem_state_adjoint -- the adjoint chain of Section 2.2 for the rigid body and
 * the cost f = 1/2 sum_m |p(x_m)|^2 over observation points, in one call:
 *   1. the state solve (1/2 I - D) p = b (GMRES, as bem_gmres_solve);
 *   2. the pressure at the observers, p(x_m) = p_inc(x_m) + (D p)(x_m) (the
 *      representation formula, bem_eval_points);
 *   3. the adjoint weights conj(p(x_m)) and the adjoint right-hand side
 *      sum_m conj(p(x_m)) G(c_i - x_m) (bem_point_sources);
 *   4. the adjoint solve with the same operator and settings.
 *   b            : [N] state right-hand side (device, dtype).
 *   observers    : [nobs][3] FP64 (device), off the surface.
 *   incident_obs : complex128 [nobs] (device), p_inc at the observers.
 *   tol, max_iter, restart, flags : as bem_gmres_solve (without
 *                  BEM_GMRES_USE_X0: both solves start from zero).
 *   p, p_adj     : [N] (device, dtype) out: the state and adjoint densities.
 *   p_obs        : complex128 [nobs] (device) out: p(x_m).
 *   weights      : complex128 [nobs] (device) out: conj(p(x_m)).
 *   iters, relres: [2] (host) out: per solve, as bem_gmres_solve.
 * Returns the first failing step's status (BEM_ERR_NOT_CONVERGED from either
 * solve, with the outputs of the steps done so far).  Synchronises `stream`
 * as the solves do; allocates (N + nobs) complex values stream-ordered.
 */
int bem_state_adjoint(bem_handle* h, int dtype, const void* b, int nobs, const double* observers,
                      const double* incident_obs, double tol, int max_iter, int restart, int flags, void* p,
                      double* p_obs, double* weights, void* p_adj, int* iters, double* relres, void* stream);

/*
 * bem_topological_field -- the topological derivative T (Section 2.5) at
 * field points from a bem_state_adjoint result, in one call:
 *   p  = p_inc + D p_surf            (state field and gradient, bem_eval_points)
 *   pa = phi + D pa_surf             (adjoint field: phi the point sources at
 *                                     the observers with the adjoint weights,
 *                                     bem_point_source_field)
 *   T  = Re[c1 grad p . grad pa - c2 p pa]   (bem_topological_derivative).
 *   p, p_adj   : [N] (device, dtype): state and adjoint densities.
 *   observers, weights : [nobs][3] FP64 and complex128 [nobs] (device).
 *   points     : [npoints][3] FP64 (device), in the fluid, off the surface.
 *   incident   : complex128 [npoints][4] (device): p_inc and its gradient.
 *   c1, c2     : as bem_topological_derivative.
 *   T          : FP64 [npoints] (device) out.
 * Allocates 4 npoints complex values in dtype and 2 x 4 npoints complex128
 * stream-ordered.  Stream-ordered; no host synchronisation.
 */
int bem_topological_field(bem_handle* h, int dtype, const void* p, const void* p_adj, int nobs,
                          const double* observers, const double* weights, int64_t npoints, const double* points,
                          const double* incident, double c1, double c2, double* T, void* stream);

/*
 * bem_levelset_step -- one step of the level-set update of Section 2.4 on a
 * lattice of n0 x n1 x n2 nodes with spacing h (the lattice that carries phi
 * and the topological derivatives):
 *   d phi / dt = F + tau L^2 lap phi,  F = -C T_omega where phi <= 0 (fluid),
 *   F = C T_omegac where phi > 0 (body),  phi = phi_bar on the lattice boundary,
 * discretised with Q1 elements on the voxels, implicit in the diffusion and
 * explicit in F:  (M / dt + tau L^2 K) phi_new = M (phi / dt + F) on the
 * interior nodes, then phi_new clamped to [-1, 1].  The interior system is
 * solved by matrix-free conjugate gradients (27-point stencil) in FP64,
 * starting from phi, to ||r|| <= tol ||rhs||.
 *   phi, t_omega, t_omegac : FP64 [n0][n1][n2] (device), node (i, j, k) at
 *                            i n1 n2 + j n2 + k.
 *   phi_out                : FP64 [n0][n1][n2] (device), may not alias phi.
 *   iters_out, relres_out  : (host, nullable) CG iterations and final relative residual.
 * Returns BEM_ERR_NOT_CONVERGED (phi_out holds the last iterate, clamped) when
 * max_iter is reached.  Allocates 9 n0 n1 n2 doubles stream-ordered and
 * synchronises `stream` every 8 iterations to read the residual.
 */
int bem_levelset_step(int n0, int n1, int n2, const double* phi, const double* t_omega, const double* t_omegac,
                      double h, double dt, double C, double tau, double L, double phi_bar, double tol, int max_iter,
                      double* phi_out, int* iters_out, double* relres_out, void* stream);

/*
 * bem_isosurface -- the boundary {phi = t} of the level-set region {phi > t}
 * as a closed triangle mesh (Section 2.4: the elastic body is where phi > 0,
 * the fluid where phi <= 0, and the boundary is phi = 0), by marching
 * tetrahedra: every grid cube splits into the 6 tetrahedra from its corner
 * (0,0,0) to (1,1,1) along the 6 axis orders; a tetrahedron with 1 or 3
 * corners inside gives one triangle, with 2 inside two.  A cut point sits on
 * its grid edge (a, b), a the lower end, at a + s (b - a) with
 * s = (t - phi_a) / (phi_b - phi_a) clamped to [0.02, 0.98], and is shared
 * by every tetrahedron around the edge, so the mesh is closed wherever the
 * region stays inside the grid.  Triangles face out of the region {phi > t}.
 *   n0, n1, n2 : grid points per axis (>= 2 each; 7 n0 n1 n2 < 2^31).
 *   phi        : FP64 [n0][n1][n2] (device); phi[i][j][k] is the value at
 *                lo + (i, j, k) h.
 *   lo         : host double[3]; h > 0; t: the level.
 *   vertices   : device FP64 [max_vertices][3], or NULL to count only.
 *   triangles  : device int32 [max_triangles][3] (a bem_mesh's layout), or
 *                NULL to count only.
 *   counts     : host int64[2]: receives the vertex and triangle counts.
 * Order: vertices by (grid point, edge direction), triangles by (cube,
 * tetrahedron, piece) -- the same for every run.  Errors: BEM_ERR_INVALID_ARG
 * when the output does not fit (counts are filled, nothing is written);
 * BEM_ERR_NUMERIC when phi holds a NaN or an infinity.  Synchronises
 * `stream`.  Keeps a grow-only device scratch of about 17 n0 n1 n2 bytes for
 * later calls; calls from several threads run one at a time.
 */
int bem_isosurface(int n0, int n1, int n2, const double* phi, const double* lo, double h, double t, double* vertices,
                   int64_t max_vertices, int* triangles, int64_t max_triangles, int64_t* counts, void* stream);

/*
 * bem_gmres_solve -- solve (1/2 I - D) x = b by restarted GMRES (Section 2.3,
 * Eq. (GMRES) without the FEM coupling term, i.e. the rigid scatterer;
 * tolerance as in Section 3).  bem_gmres_solve_coupled adds the term.
 *   b          : right-hand sides [nrhs][N] (device).
 *   x          : in: initial guess if (flags & BEM_GMRES_USE_X0) else ignored;
 *                out: solution [nrhs][N] (device).
 *   tol        : stop when ||b - A x||_2 / ||b||_2 <= tol for every rhs
 *                (recursive residual).
 *   max_iter   : total iteration cap; restart: Krylov dimension per cycle.
 *   iters_out  : nullable; receives the iterations used.
 *   relres_out : nullable host array [nrhs]; receives the final relative residuals.
 *   flags      : BEM_GMRES_USE_X0; BEM_GMRES_HOST_LOOP runs the Arnoldi steps
 *                from the host; BEM_GMRES_GRAPH_ONLY makes a failure to build
 *                the graph an error instead of falling back to the host loop.
 * Orthogonalisation is classical Gram-Schmidt applied twice, in FP64.
 * Returns BEM_ERR_NOT_CONVERGED (with x = last iterate) if max_iter is reached.
 * By default every restart cycle is one CUDA graph (built once per call):
 * the Arnoldi steps run in a conditional WHILE node, the Givens rotations of
 * the small least-squares problems run on the device, and `stream` is
 * synchronised once per cycle to read the residuals.  The host loop
 * synchronises once per iteration.  The call allocates about
 * (min(restart, max_iter) + 5) * nrhs * N * 16 bytes of stream-ordered
 * scratch for its Krylov basis and frees it before returning.
 */
#define BEM_GMRES_USE_X0 1
#define BEM_GMRES_HOST_LOOP 2
#define BEM_GMRES_GRAPH_ONLY 4
int bem_gmres_solve(bem_handle* h, int nrhs, int dtype, const void* b, void* x, double tol, int max_iter, int restart,
                    int flags, int* iters_out, double* relres_out, void* stream);

/*
 * bem_coupling_fn -- the caller's coupling map of Eq. (GMRES): on entry `cx`
 * (the buffer given to bem_gmres_solve_coupled) holds a vector x, complex128
 * [nrhs][N], written in stream order on `stream`; the callback must leave
 * y = C x in `cy` in stream order on `stream` (enqueue its work there, or
 * finish it and synchronise) and return 0.  For the BEM-FEM system of
 * Section 2.3, C = T (K - rho_s omega^2 M)^{-1} N: N maps the pressure to
 * nodal loads, the factorised FEM matrix gives the displacement, and T maps
 * it to the normal-derivative density that the single layer S acts on.
 * Any non-zero return ends the solve with BEM_ERR_CALLBACK.
 */
typedef int (*bem_coupling_fn)(void* ctx, int nrhs, void* stream);

/*
 * bem_gmres_solve_coupled -- solve (1/2 I - D + S C) x = b (Eq. (GMRES),
 * Section 2.3) by restarted GMRES.  Every matrix-vector product is step 2 of
 * the paper's algorithm: the callback computes y = C x (steps 2(a) and 2(b)),
 * then one FMM apply gives (1/2 I - D) x + S y (step 2(c)).
 *   cb, cb_ctx : the coupling map (non-NULL) and its context.
 *   cx, cy     : caller-owned device buffers, complex128 [nrhs][N] each,
 *                16-byte aligned, not overlapping b, x or each other.  Their
 *                addresses stay fixed for the whole call, so the callback may
 *                prepare its work on them once.
 *   other arguments as for bem_gmres_solve.
 * The Arnoldi steps run from the host (the callback is arbitrary host code,
 * which stream capture cannot hold): BEM_GMRES_HOST_LOOP is implied and
 * BEM_GMRES_GRAPH_ONLY returns BEM_ERR_UNSUPPORTED.
 */
int bem_gmres_solve_coupled(bem_handle* h, int nrhs, int dtype, const void* b, void* x, double tol, int max_iter,
                            int restart, bem_coupling_fn cb, void* cb_ctx, double* cx, double* cy, int flags,
                            int* iters_out, double* relres_out, void* stream);

/*
 * The elastic body of Section 2.3 (the FEM half of the coupled solver).
 *
 * bem_fem_setup -- P1 tetrahedra of the body Omega^c: K - rho_s omega^2 M is
 * assembled and factorised on the GPU (step 1 of the paper's algorithm).
 *   nodes  : [n_nodes][3] FP64 node coordinates (host).
 *   tets   : [n_tets][4] int32 node indices (host), either orientation.
 *   tris   : [n_tris][3] int32 node indices (host): the boundary faces of the
 *            tetrahedra, i.e. the BEM mesh, ordered so that the normal points
 *            out of the body (the BEM operator of the same triangles and the
 *            same node array gives S and D of Eq. (GMRES)).
 *   lambda, mu : Lame constants (mu > 0, 3 lambda + 2 mu > 0); rho_s, rho_f:
 *            solid and fluid densities; omega: angular frequency.
 *   flags  : BEM_FEM_KEEP_MATRIX keeps a copy of the assembled matrix for
 *            bem_fem_matrix.
 * Element matrices as in the Galerkin form of Section 2.3 with the isotropic
 * C_ijkl: K_e[(a,i),(b,k)] = V (lambda g_ai g_bk + mu g_ak g_bi + mu delta_ik
 * g_a.g_b), M_e = delta_ik V (1 + delta_ab) / 20; degrees of freedom 3 a + i.
 * The matrix is held dense (FP64, (3 n_nodes)^2 * 8 bytes, at most 60,000
 * degrees of freedom) and factorised by LU with partial pivoting; the paper
 * uses a sparse multifrontal solver.  Fails with BEM_ERR_INVALID_ARG on a
 * node index out of range, a degenerate tetrahedron or triangle, or a
 * singular matrix (omega^2 an eigenvalue of the free body).
 */
typedef struct bem_fem bem_fem;
#define BEM_FEM_KEEP_MATRIX 1
int bem_fem_setup(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets, const int32_t* tris,
                  int64_t n_tris, double lambda, double mu, double rho_s, double rho_f, double omega, int flags,
                  void* stream, bem_fem** out);
int bem_fem_destroy(bem_fem* f);

/* u = (K - rho_s omega^2 M)^{-1} b for nrhs (1..64) real columns b, u
 * [nrhs][3 n_nodes] (device, FP64), in stream order. */
int bem_fem_solve(bem_fem* f, int nrhs, const double* b, double* u, void* stream);

/*
 * bem_fem_couple -- y = C x, the coupling map of Eq. (GMRES) (steps 2(a) and
 * 2(b) of the paper's algorithm), for complex element pressures x and
 * densities y [nrhs][n_tris] (nrhs 1..32) in dtype (device), in stream order:
 *   C = rho_f omega^2 Avg (K - rho_s omega^2 M)^{-1} (-N),
 * N[(a,i), j] = n_ji A_j / 3 the load of a unit pressure on triangle j (the
 * traction is -p n by the boundary condition t_i + p n_i = 0), Avg[j, (a,i)]
 * = n_ji / 3 the element mean of u.n: the single layer then takes
 * q = rho_f omega^2 u.n as its density, so (1/2 I - D + S C) p = p_src.
 */
int bem_fem_couple(bem_fem* f, int nrhs, int dtype, const void* x, void* y, void* stream);

/* bem_fem_bind / bem_fem_coupling -- the coupling map as a bem_coupling_fn:
 * bind the complex128 buffers cx, cy given to bem_gmres_solve_coupled, then
 * pass bem_fem_coupling with ctx = f, so that the whole coupled solve runs in
 * the library. */
int bem_fem_bind(bem_fem* f, const void* cx, void* cy);
int bem_fem_coupling(void* ctx, int nrhs, void* stream);

/* the assembled K - rho_s omega^2 M, column-major [3 n_nodes][3 n_nodes] FP64,
 * into a host or device buffer (requires BEM_FEM_KEEP_MATRIX). */
int bem_fem_matrix(bem_fem* f, double* out, void* stream);

enum {
  BEM_FEM_INFO_DOF = 0,   /* 3 n_nodes */
  BEM_FEM_INFO_NODES = 1,
  BEM_FEM_INFO_TETS = 2,
  BEM_FEM_INFO_TRIS = 3,
  BEM_FEM_INFO_BYTES = 4  /* device bytes held */
};
int bem_fem_info(bem_fem* f, int key, int64_t* value);

/*
 * Batches of independent problems (many scatterers, each with its own mesh
 * and wavenumber: the state and adjoint solves of Section 2.5 repeated over a
 * population of designs).  Every problem keeps its own octree and operators;
 * a batch apply runs all of them from one captured CUDA graph whose branches
 * (problems spread over up to 64 forked streams) execute concurrently.
 */
typedef struct bem_batch bem_batch;

/*
 * bem_setup_batch -- bem_setup for `count` meshes with wavenumbers ks[count]
 * (same p, eps and options for all).  Synchronises `stream`.
 */
int bem_setup_batch(const bem_mesh* meshes, const double* ks, int count, int p, double eps, const bem_options* opt,
                    void* stream, bem_batch** out);

/*
 * bem_setup_batch_each -- bem_setup_batch with options per problem:
 *   opts : count bem_options (each with its own struct_size; not nullable),
 *          e.g. the tree and tile choices an autotuner made for each body.
 * Every problem must use the same max_nrhs.
 */
int bem_setup_batch_each(const bem_mesh* meshes, const double* ks, int count, int p, double eps,
                         const bem_options* opts, void* stream, bem_batch** out);

/*
 * bem_apply_batch -- z = (1/2 I - D) x + S y for every problem at once.
 *   x, y, z : device buffers [nrhs][N_total] where N_total is the sum of the
 *             problems' triangle counts; problem b owns the columns
 *             [N_0 + ... + N_{b-1}, + N_b) of every rhs row.
 *   flags   : BEM_APPLY_NO_HALF.
 * The first call for a given (nrhs, flags) captures the graph (host work);
 * later calls are two small staging kernels and one graph launch on `stream`.
 */
int bem_apply_batch(bem_batch* b, int nrhs, int dtype, const void* x, const void* y, void* z, int flags, void* stream);

/*
 * bem_batch_info -- problem = -1: key 0 -> N_total, key 1 -> number of
 * problems; problem >= 0: bem_info of that problem's handle.
 */
int bem_batch_info(bem_batch* b, int problem, int key, int64_t* value);

/*
 * bem_gmres_solve_batch -- bem_gmres_solve for every problem of a batch at
 * once: (1/2 I - D_p) x_p = b_p for every problem p and right-hand side.
 *   rhs, x     : [nrhs][N_total] device buffers in the batch's concatenated
 *                layout (problem p owns its contiguous segment of each rhs).
 *   relres_out : nullable host array [nrhs][number of problems].
 * Every (rhs, problem) segment is its own GMRES system with its own Krylov
 * space, tolerance test and residual; all of them advance in lockstep, and
 * each iteration is one bem_apply_batch of the whole batch.  iters_out gets the
 * lockstep iteration count (the largest over the systems).  Other arguments,
 * the errors and the scratch are as for bem_gmres_solve with N = N_total.
 */
int bem_gmres_solve_batch(bem_batch* b, int nrhs, int dtype, const void* rhs, void* x, double tol, int max_iter,
                          int restart, int flags, int* iters_out, double* relres_out, void* stream);

/* bem_destroy_batch -- free a batch and every handle in it (NULL accepted). */
int bem_destroy_batch(bem_batch* b);

/*
 * bem_info -- integer facts about a handle (sizes, counts, orders), for
 * reporting and for the roofline arithmetic.  Unknown keys -> INVALID_ARG.
 */
typedef enum {
  BEM_INFO_N = 0,            /* triangles */
  BEM_INFO_LEAF_LEVEL = 1,    /* deepest level of the octree (the leaf level of a uniform tree) */
  BEM_INFO_N_LEAVES = 2,      /* leaves over all levels */
  BEM_INFO_P2P_PAIRS = 3,    /* (target, source triangle) pairs of the near field */
  BEM_INFO_CORR_NNZ = 4,     /* entries of the near-singular correction matrix */
  BEM_INFO_M2L_PAIRS = 5,    /* V-list pairs over all levels */
  BEM_INFO_M2L_FLOPS = 6,    /* 8 P_l^2 per V-list pair summed over levels (one rhs) */
  BEM_INFO_P_LEAF = 7,       /* expansion order at the deepest level */
  BEM_INFO_P_TOP = 8,        /* expansion order at level 2 */
  BEM_INFO_MODE = 9,
  BEM_INFO_DEVICE_BYTES = 10,
  BEM_INFO_P2M_BYTES = 11,   /* bytes of the stored P2M + L2P rows */
  BEM_INFO_LAUNCHES_LAST_APPLY = 12, /* kernels the last bem_apply launched (memsets excluded) */
  BEM_INFO_M2M_FLOPS = 13,   /* 8 P_child P_parent per child box summed over levels (one rhs) */
  BEM_INFO_L2L_FLOPS = 14,   /* 8 P_parent P_child per child box summed over levels (one rhs) */
  BEM_INFO_ADAPTIVE = 15,    /* 0: uniform tree, 1: per-region depth (leaf_level -1), 2: per-box split (-2) */
  BEM_INFO_ROW_COEFFS = 16,  /* coefficients of the stored L2P rows over all elements (P2M rows: twice as many) */
  BEM_INFO_W_PAIRS = 17,     /* (target leaf, source box) pairs of the W-lists (M2P) */
  BEM_INFO_X_PAIRS = 18,     /* (target box, source leaf) pairs of the X-lists (P2L) */
  BEM_INFO_NEAR_LIST = 19,   /* entries of the near-field (U-) lists over all leaves */
  BEM_INFO_W_EVALS = 20,     /* (target, coefficient) products of the M2P work (one rhs) */
  BEM_INFO_X_EVALS = 21,     /* (source point, coefficient) products of the P2L work (one rhs) */
  BEM_INFO_EXP_TOTAL = 22,   /* expansion coefficients per rhs over all levels (the far-field buffers' length) */
  BEM_INFO_TC_KIND = 23,     /* tensor-core translations: 0 none (FP64 or direct modes), 1 FP16 split, 2 3xTF32, 3 plain TF32 */
  BEM_INFO_ORDER_OF_LEVEL = 100, /* + level: expansion order of that level */
  BEM_INFO_LEAVES_OF_LEVEL = 200, /* + level: leaves on that level */
  BEM_INFO_BOXES_OF_LEVEL = 300,  /* + level: occupied boxes on that level (tree or not) */
  BEM_INFO_EXP_BASE_OF_LEVEL = 400 /* + level: first coefficient of that level's expansions */
} bem_info_key;
int bem_info(bem_handle* h, int key, int64_t* value);

/*
 * Inspection of the octree and of the FMM stages (Section 2.3's far field),
 * so that each translation can be checked against direct sums.  Not needed to
 * apply or solve; every call synchronises.
 *
 * bem_tree_level -- the occupied boxes of one level (0 .. BEM_INFO_LEAF_LEVEL),
 * in Morton order, BEM_INFO_BOXES_OF_LEVEL + level of them.  Host buffers,
 * each nullable: start/end [nbox] element range in sorted order (see
 * bem_sorted_order), centre [nbox][3], flags [nbox] (bit 0: the box is in the
 * tree, bit 1: it is split; a tree box that is not split is a leaf).
 */
int bem_tree_level(bem_handle* h, int level, int* start, int* end, double* centre, unsigned char* flags);

/* bem_sorted_order -- perm[s] = caller index of the element at sorted position s (host buffer [N]). */
int bem_sorted_order(bem_handle* h, int* perm);

/*
 * bem_far_field -- run one apply of x, y (as bem_apply, device buffers) and
 * return its far-field intermediates in textbook normalisation (FMM modes only):
 *   M    : [nrhs][E] complex128 multipoles, u(x) = sum_nm M_nm h_n(k|x-c|) Y_nm
 *          about each box centre c (E = BEM_INFO_EXP_TOTAL; box b of level l at
 *          BEM_INFO_EXP_BASE_OF_LEVEL + l + b (p_l + 1)^2, coefficient n^2+n+m);
 *   L    : [nrhs][E] complex128 local expansions, u(x) = sum_nm L_nm j_n(k|x-c|) Y_nm,
 *          after the downward pass (before L2P);
 *   zfar : [nrhs][N] complex128 far-field part of z in the caller's order.
 * Y_nm is orthonormal without the Condon-Shortley phase, Y_n,-m = conj(Y_nm).
 * Device buffers, each nullable.  Synchronises `stream`.
 */
int bem_far_field(bem_handle* h, int nrhs, int dtype, const void* x, const void* y, double* M, double* L,
                  double* zfar, void* stream);

/*
 * bem_profile -- per-stage device timing of bem_apply (measurement support for
 * the stage breakdown the paper reports as Table 2, here at kernel level).
 *   enable = 1: from now on every bem_apply records a pair of CUDA events
 *               around each stage on the caller's stream (about 1 us each).
 *   enable = 0: stop recording.  Either value synchronises the device and
 *               discards the records collected so far.
 * Stages: 0 prologue, 1 P2P near field, 2 near-singular correction, 3 P2M,
 * 4 M2M, 5 M2L, 6 L2L, 7 L2P, 8 epilogue.
 */
int bem_profile(bem_handle* h, int enable);

/*
 * bem_profile_read -- wait for the recorded events and return, per stage,
 * the summed device milliseconds (ms[nstages]) and the number of kernel
 * launches (launches[nstages], nullable) since the last bem_profile call.
 */
int bem_profile_read(bem_handle* h, double* ms, int64_t* launches, int nstages);

/*
 * bem_last_error -- message of the last failing call on this thread ("" if none).
 */
const char* bem_last_error(void);

/*
 * bem_sync -- synchronise `stream` and report the device-side problem flags
 * that kernels of this handle raised since the last synchronising call
 * (bem_apply, bem_apply_adjoint and bem_eval_points are stream-ordered and
 * return before their kernels run, so this is where their device-side errors
 * surface): BEM_ERR_TIMEOUT when a bounded device wait expired, BEM_ERR_NUMERIC
 * for non-finite values.  The flags are cleared when read.  (Section 8(b) error
 * contract; the paper has no counterpart.)
 */
int bem_sync(bem_handle* h, void* stream);

/*
 * bem_set_wait_limit -- diagnostic of the bounded-wait path (no counterpart in
 * the paper).  Every mbarrier wait of the tensor-core translations gives up
 * after a bounded number of SM clocks, sets a device flag, waits (bounded) for
 * its own copies and MMAs, frees its tensor memory and returns, so no kernel of
 * this library can wait forever.
 *   clocks : bound of the main-loop wait for a translation-matrix stage, in SM
 *            clocks; <= 0 restores the default 2^31 (about one second).  The
 *            drain waits at the end of a CTA keep the default bound.
 *   hold   : != 0 makes every translation CTA withhold its first matrix copy,
 *            so its first wait expires with nothing in flight; 0 restores the
 *            normal path.
 * With hold set, the next FMM apply in the mixed or tf32 mode produces a wrong
 * far field and bem_sync returns BEM_ERR_TIMEOUT; the handle stays usable.
 * For tests of the timeout path only.
 */
int bem_set_wait_limit(bem_handle* h, long long clocks, int hold);

/*
 * bem_peak_probe -- microbenchmark of a compute pipe, for roofline
 * denominators that no vendor figure fixes on this part (the paper has no
 * counterpart; it is a measuring tool of this library).
 *   which  : 0 = FP32 through packed f32x2 FMAs (8 independent chains per
 *            thread, 8 blocks of 256 threads per SM);
 *            1 = dense TF32 through tcgen05.mma (M = 128, N = 256, K = 8,
 *            operands resident in shared memory, one TMEM accumulator per CTA,
 *            2 CTAs per SM);
 *            2 = dense FP16 through tcgen05.mma kind::f16 (K = 16, same shape and
 *            residency), the rate of the FP16-split translations.
 *   iters  : iterations per thread (0) or MMAs per CTA (1), 1 .. 2^20.
 *   tflops : receives the rate of the second of two launches, in TFLOP/s
 *            (an FMA counts 2 flops).
 * Allocates two small stream-ordered buffers and synchronises `stream`.
 * A bounded device wait that expires returns BEM_ERR_TIMEOUT.
 */
int bem_peak_probe(int which, int iters, double* tflops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* BEM_H_ */
