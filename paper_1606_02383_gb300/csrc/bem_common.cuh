// bem_common.cuh -- shared types of the GB300 BEM/FMM library (device + host).
//
// Layout of the handle's device state (all per-element arrays are in octree
// (Morton) order; perm[s] maps a sorted index s to the caller's index):
//   geometry   : centroids, quadrature points, normals, areas, longest edges
//   octree     : per level l = 0..L the occupied boxes (Morton prefix, element
//                range, parent, first child, child count, integer coordinates)
//   lists      : 27-slot colleague table of every leaf (near field), V-list
//                pairs grouped by (level, offset), M2M/L2L pairs grouped by octant
//   operators  : scaled translation matrices per (level, offset/octant), P2M
//                and L2P rows per element, near-singular correction in CSR
//   workspaces : weighted densities, multipole/local expansions, partial sums
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/bem.h"

#define BEM_MAXLEV 10  // Morton keys carry 10 bits per axis
#define BEM_PI 3.14159265358979323846

// ---------------------------------------------------------------- complex --
template <typename R>
struct cpx {
  R re, im;
};
template <typename R>
__host__ __device__ __forceinline__ cpx<R> cmk(R a, R b) {
  cpx<R> c;
  c.re = a;
  c.im = b;
  return c;
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) {
  return cmk(a.re + b.re, a.im + b.im);
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) {
  return cmk(a.re - b.re, a.im - b.im);
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator*(cpx<R> a, cpx<R> b) {
  return cmk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator*(R s, cpx<R> a) {
  return cmk(s * a.re, s * a.im);
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> conjc(cpx<R> a) {
  return cmk(a.re, -a.im);
}
typedef cpx<double> zd;
typedef cpx<float> zf;

// i^n for integer n
__host__ __device__ __forceinline__ zd ipow(int n) {
  int m = ((n % 4) + 4) % 4;
  return m == 0 ? cmk(1.0, 0.0) : m == 1 ? cmk(0.0, 1.0) : m == 2 ? cmk(-1.0, 0.0) : cmk(0.0, -1.0);
}

// ------------------------------------------------------------ status codes --
struct BemError {
  int code;
  std::string msg;
};

void bem_set_error(const std::string& m);
int bem_fail(int code, const std::string& m);

#define BEM_CUDA(call)                                                                          \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return bem_fail(e_ == cudaErrorMemoryAllocation ? BEM_ERR_OOM : BEM_ERR_CUDA,             \
                      std::string(#call) + ": " + cudaGetErrorString(e_));                      \
  } while (0)

#define BEM_TRY(call)            \
  do {                           \
    int rc_ = (call);            \
    if (rc_ != BEM_OK) return rc_; \
  } while (0)

// Device-side problem flags (written by kernels, read at synchronising calls).
#define BEM_DEVERR_DEGENERATE 1
#define BEM_DEVERR_NONFINITE 2
#define BEM_DEVERR_OVERFLOW 4
#define BEM_DEVERR_TIMEOUT 8

// Signed permutation of a reflection (flags: bit 0 = x, 1 = y, 2 = z) acting on
// the coefficient index k = n^2 + n + m of an expansion: an x or y flip maps
// m -> -m (both together cancel), an x flip contributes (-1)^m and a z flip
// (-1)^(n+m).  Returns the permuted index and sets *neg for a sign change.
__device__ __forceinline__ int reflect_index(int k, int flags, bool* neg) {
  int n = (int)sqrtf((float)k);
  if ((n + 1) * (n + 1) <= k) ++n;
  if (n * n > k) --n;
  int m = k - n * n - n;
  bool s = ((flags & 1) && (m & 1)) != ((flags & 4) && ((n + m) & 1));
  *neg = s;
  return (((flags & 1) != 0) != ((flags & 2) != 0)) ? (n * n + n - m) : k;
}

// ------------------------------------------------------------------ handle --
struct GroupedOp {
  int upward = 0;  // 1: an M2M (child to parent) operator, few long jobs per level
  // For every pair c of group g, with Q_c the signed permutation of the pair's
  // reflection flags (x, y, z bits):
  //   dst[dst_off[c] + .] += Q_c T_g Q_c src[src_off[c] + .]
  // T_g is the translation matrix of the group's canonical vector (all
  // components >= 0); a reflected vector R v gives T(R v) = Q T(v) Q.
  int ngroups = 0;
  std::vector<int> rows, cols;          // per group (host copy)
  std::vector<int64_t> mat_off;         // per group, complex offset into the matrix buffer
  std::vector<int> pair_start;          // per group, first pair (host copy), size ngroups+1
  std::vector<int> codes;               // tree build: offset code of every V-list group
  const void* mats_base = nullptr;      // matrix buffer the group offsets refer to
  int npairs = 0;
  int* d_src_off = nullptr;             // [npairs]
  int* d_dst_off = nullptr;             // [npairs]
  unsigned char* d_flags = nullptr;     // [npairs] reflection bits
  // tile jobs: (group, first pair, npairs | k-slice << 8, row0); A = 64x64 tiles, B = 128x16 tiles;
  // K is split into slices of 128 (outputs are accumulated atomically anyway)
  int njobsA = 0, njobsB = 0;
  int4* d_jobsA = nullptr;
  int4* d_jobsB = nullptr;
  int* d_group_rows = nullptr;
  int* d_group_cols = nullptr;
  int64_t* d_group_mat = nullptr;
  int64_t flops = 0;                    // 8 * rows * cols per pair, summed
  // tensor-core form (mixed mode): A packed per (row tile, k stage), jobs (group, pair0, npairs, row tile)
  // source level of the pairs (its expansions are prepared, reflected and split, before every launch)
  int src_level = -1;
  int tc_kslice = 16;  // K stages per tensor-core job
  // a second job list with shorter K slices, for launches with too few CTAs
  // for the SMs (small operators at one right-hand side)
  int4* d_tc_jobs_split = nullptr;
  int n_tc_jobs_split = 0;
  int tc_kslice_split = 16;
  int64_t tc_want = 0;  // CTAs that give every SM two
  int* d_prep_row = nullptr;            // [npairs] row (flag * nbox + box) of the prepared source
  int* d_prep_list = nullptr;           // [n_prep_list] distinct rows the pairs read (when few)
  int n_prep_list = 0;
  float* tcA = nullptr;
  float* tscale = nullptr;  // FP16 split: inverse power-of-two scale of every matrix row, per group at d_tsoff[g]
  int* d_tsoff = nullptr;
  int64_t* d_tc_off = nullptr;
  int4* d_tc_jobs = nullptr;
  int n_tc_jobs = 0;
};


struct LevelInfo {
  int nbox = 0;
  int p = 0, P = 0;
  double w = 0.0;        // box width
  int64_t exp_base = 0;  // complex offset of this level's expansions within one rhs slab
  // device arrays (per box)
  uint32_t* key = nullptr;  // Morton prefix of the box
  int* start = nullptr;     // first element (sorted order)
  int* end = nullptr;       // one past last element
  int* child0 = nullptr;    // first child box (level l+1), -1 at the leaf level
  int* nchild = nullptr;
  int* parent = nullptr;    // parent box (level l-1), -1 at the root
  int* coord = nullptr;     // [nbox][3] integer box coordinates at this level
  double* centre = nullptr; // [nbox][3]
  // tree membership (adaptive octree): a box is in the tree when its parent is
  // an internal tree box; a tree box is a leaf or internal
  unsigned char* intree = nullptr;    // [nbox]
  unsigned char* internal = nullptr;  // [nbox]
  int nleaf = 0;                      // leaves on this level
  int* leafbox = nullptr;             // [nleaf] box index of every leaf of this level
  int leaf_g0 = 0;                    // global index of this level's first leaf
  float* gap2 = nullptr;              // [nbox] (4 h_max(box) / w_L)^2, the off-surface walk's far test
};

// per-level orders and expansion offsets, passed by value to kernels that
// handle elements or boxes of several levels
struct LevTab {
  int P[BEM_MAXLEV + 1];
  long long base[BEM_MAXLEV + 1];
};

// one profiled stage of one apply: events recorded on the caller's stream
struct ProfRec {
  int stage;
  cudaEvent_t a, b;
  int launches;
};
#define BEM_NSTAGES 9  // prologue, p2p, correction, p2m, m2m, m2l, l2l, l2p, epilogue

struct bem_handle {
  int device = 0;
  int mode = BEM_MODE_FMM_MIXED;
  double k = 0.0;
  int fixed_p = 0;
  double eps = 1e-5;
  int nrhs_max = 16;
  int p2p_unit = 64;       // most targets per near-field warp work unit
  int tc_kslice_max = 16;  // most K stages per tensor-core translation job
  int corr_rules32 = 0;    // mixed modes: non-self near-singular rules summed in FP32
  int tc_fp16 = 0;   // mixed mode: translations as the FP16 split (else 3xTF32)
  int tc_pipeline = 0;  // translation kernel: 0 per operator (M2M persistent, others 2 stages),
                        // 1 block-synchronous, 2 / 4 warp-specialised stages, 3 persistent
  int p2p_ctas = 0;     // > 0: near field from this many resident CTAs per SM, beside the far field
  int p2p_stage = 0;    // 1: near-list elements staged in shared memory by cp.async chunks
  int grad_direct = 0;  // 1: the vertex gradient's regular rule as an all-pairs sum on FMM handles
  int nsm = 0;          // SMs of the device
  int* p2p_ctr = nullptr;  // [nrhs_max + 2] unit counters of the resident near field
  int p_min = 4, p_max = 40;
  int p_level[BEM_MAXLEV + 1] = {0};  // explicit per-level orders (0 = automatic)
  int64_t nt = 0, nv = 0;
  int L = 0;          // leaf level
  int Lc = 0;         // level used to search for near-singular pairs
  double root_c[3] = {0, 0, 0};
  double root_w = 0;  // root box width
  std::vector<LevelInfo> lev;

  std::vector<void*> allocs;  // everything cudaMalloc'ed for this handle
  size_t bytes = 0;

  int* d_err = nullptr;  // device problem flags

  // geometry (sorted order)
  int* perm = nullptr;          // sorted -> caller index
  double* cent = nullptr;       // [nt][3]
  double* qpt = nullptr;        // [nt][3][3]
  double* nrm = nullptr;        // [nt][3]
  double* area = nullptr;       // [nt]
  double* hmax = nullptr;       // [nt]
  double* wgt = nullptr;        // A_j / (12 pi): quadrature weight per point, with 1/(4 pi)
  int* tri = nullptr;           // [nt][3] caller's vertex indices of every sorted element
  float4* tgt32 = nullptr;      // [nt] centroid
  float4* src32 = nullptr;      // [nt][3] quadrature points, normal in .w
  double4* tgt64 = nullptr;
  double4* src64 = nullptr;
  double hmax_all = 0.0;

  // octree leaves.  A fixed leaf level (bem_options.leaf_level > 0) gives a
  // uniform tree; otherwise boxes are split while they hold more than the
  // split threshold and their children stay at least 3 longest edges wide, so
  // leaves sit on several levels.  Global leaf g covers elements
  // [gl_start[g], gl_end[g]); leaves are numbered level by level.
  int adaptive = 0;
  int nleaf_all = 0;
  int* gl_start = nullptr;      // [nleaf_all]
  int* gl_end = nullptr;        // [nleaf_all]
  int* leaf_of = nullptr;       // [nt] box (within its level) of every element's leaf
  unsigned char* leaf_lev = nullptr;  // [nt] level of every element's leaf
  int* gleaf_of = nullptr;      // [nt] global leaf of every element
  // P2M and L2P rows: element j's rows start at coefficient row_off[j] (P of
  // its leaf level, rounded up to even, per element): P2M at 2 row_off[j],
  // L2P at row_off[j] (complex units)
  int64_t* row_off = nullptr;
  int64_t row_total = 0;
  // near field (U-lists): for leaf g, entries [u_ptr[g], u_ptr[g+1]): every
  // leaf adjacent to g (any level, g itself included), with the offset
  // centre(source leaf) - centre(g)
  int* u_ptr = nullptr;
  int* u_src = nullptr;
  float4* u_shift32 = nullptr;
  double4* u_shift64 = nullptr;
  int64_t u_nnz = 0;
  int64_t p2p_pairs = 0;
  int4* p2p_units = nullptr;    // warp work units (global leaf, first target, count), largest first
  int n_p2p_units = 0;
  // W-lists (M2P): for leaf g, entries [w_ptr[g], w_ptr[g+1]) name boxes D
  // (level << 24 | box) finer than g whose multipoles converge at g's targets,
  // with the offset centre(g) - centre(D); w_leaves lists the leaves whose
  // W-list is not empty
  int* w_ptr = nullptr;
  int* w_src = nullptr;
  float4* w_shift32 = nullptr;
  double4* w_shift64 = nullptr;
  int w_nnz = 0;
  int* w_leaves = nullptr;
  int n_w_leaves = 0;
  // X-lists (P2L), the duals of the W-lists: pairs (box B of level l, source
  // leaf C) with C's elements expanded about B's centre; offsets centre(C) -
  // centre(B)
  int x_n[BEM_MAXLEV + 1] = {0};
  int* x_dst[BEM_MAXLEV + 1] = {nullptr};
  int* x_src[BEM_MAXLEV + 1] = {nullptr};
  float4* x_shift32[BEM_MAXLEV + 1] = {nullptr};
  double4* x_shift64[BEM_MAXLEV + 1] = {nullptr};
  int64_t w_tp[BEM_MAXLEV + 1] = {0};  // (target, W box) pairs by the box's level
  int64_t x_pts[BEM_MAXLEV + 1] = {0}; // (source point, X box) pairs by the box's level
  int64_t w_evals = 0, x_evals = 0;    // (point, coefficient) products per rhs of the M2P and P2L work
  int* wx_p = nullptr;                 // [BEM_MAXLEV + 1] order of every level
  void* wx_a = nullptr;                // [BEM_MAXLEV + 1] k w_l in the operator's precision

  // correction CSR over sorted targets; values divided by wgt[j]
  int* corr_ptr = nullptr;      // [nt+1]
  int* corr_col = nullptr;      // [nnz]
  void* corr_val = nullptr;     // [nnz] of {S, D} complex (float4 or double4)
  int64_t corr_nnz = 0;
  // the correction's transpose (columns -> rows), built with the adjoint operators
  int* corrT_ptr = nullptr;     // [nt+1]
  int* corrT_row = nullptr;     // [nnz]
  void* corrT_val = nullptr;    // [nnz], same type as corr_val

  // far field
  GroupedOp m2m[BEM_MAXLEV + 1];  // index l: child level l+1 -> parent level l
  GroupedOp m2l[BEM_MAXLEV + 1];
  GroupedOp l2l[BEM_MAXLEV + 1];  // index l: parent level l -> child level l+1
  void* mats = nullptr;           // all translation matrices (complex float or double)
  int64_t mats_len = 0;
  void* p2m_rows = nullptr;       // [nt][2][P_L] complex: a-hat, b-hat
  void* l2p_rows = nullptr;       // [nt][P_L] complex
  int64_t exp_total = 0;          // complex coefficients per rhs over all levels

  // adjoint (conjugate-transpose) apply, built on first use
  bool adj_ready = false;
  GroupedOp m2m_T[BEM_MAXLEV + 1];  // index l: parent level l -> child level l+1 (transpose of m2m[l])
  GroupedOp m2l_T[BEM_MAXLEV + 1];  // target level-l Lambda -> source level-l Mu (transpose of m2l[l])
  GroupedOp l2l_T[BEM_MAXLEV + 1];  // child level l+1 -> parent level l (transpose of l2l[l])
  void* mats_T = nullptr;
  float* prep = nullptr;            // reflected, TF32- or FP16-split source expansions of one level (tensor-core path)
  int64_t prep_len = 0;
  float* prep_scale = nullptr;      // FP16 split: inverse power-of-two scale of every prepared row
  int64_t prep_scale_len = 0;
  double4* uv = nullptr;            // [nrhs_max][nt]: (u = S^T h, v = D^T h) before the weight, sorted

  // workspaces
  void* dens = nullptr;     // [nrhs_max][nt] weighted (y, x) pairs: float4 or double4
  void* Mexp = nullptr;     // [nrhs_max][exp_total] complex
  void* Lexp = nullptr;
  double* zn = nullptr;     // [nrhs_max][nt] complex double (near + correction), sorted
  double* zfar = nullptr;   // [nrhs_max][nt] complex double (far), sorted
  void* io_x = nullptr;     // staging for BEM_HOST_BUFFERS: [nrhs_max][nt] complex double each
  void* io_y = nullptr;
  void* io_z = nullptr;
  // the far field's high-priority stream, forked after the P2P and joined back
  cudaStream_t s_far = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // profiling
  int prof_on = 0;
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> ev_pool;
  int launches_last_apply = 0;  // kernels launched by the last bem_apply
  // bound of the tensor-core translations' main-loop matrix-stage wait, in SM
  // clocks, and the diagnostic that withholds every CTA's first matrix copy so
  // that this wait expires (bem_set_wait_limit)
  long long tc_wait_limit = 1LL << 31;
  int tc_hold_first_copy = 0;
};

int bem_prof_begin(bem_handle* h, cudaStream_t s);                      // returns a record index or -1
void bem_prof_end(bem_handle* h, int rec, int stage, int launches, cudaStream_t s);
bool bem_is_fmm(const bem_handle* h);
bool bem_is_fp64(const bem_handle* h);
// n-point Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n), host side
void bem_gl_host(int n, double* x, double* w);
// vertex gradient of the loss (bem_grad_vertices.cu); yx, gs: unweighted
// densities (y, x) and the upstream gradient in octree order, FP64;
// dvertices: nullable host array [nv][3], written when `s` completes;
// dk: nullable device double to which the regular-rule part of dL/dk is added
int bem_grad_vertices(bem_handle* h, int nrhs, const double4* yx, const double2* gs, double* dvertices, double* dk,
                      cudaStream_t s);

template <typename T>
int bem_alloc(bem_handle* h, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return bem_fail(BEM_ERR_OOM, std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) +
                                     " bytes failed: " + cudaGetErrorString(e));
  }
  h->allocs.push_back((void*)*p);
  h->bytes += count * sizeof(T);
  return BEM_OK;
}

// ---- stage entry points (defined in the .cu files) ----
int bem_build_geometry(bem_handle* h, const double* dV, const int32_t* dT, cudaStream_t s);
int bem_build_tree(bem_handle* h, int leaf_level, int leaf_target, cudaStream_t s);
LevTab bem_levtab(const bem_handle* h);
// W- and X-list work (bem_wx.cu): M2P into the far sums, P2L into the local
// expansions, and their transposes for the adjoint apply
int bem_build_wx_tables(bem_handle* h, cudaStream_t s);
int bem_run_m2p(bem_handle* h, int nrhs, const void* M, double* zfar, cudaStream_t s, int* launches);
int bem_run_p2l(bem_handle* h, int nrhs, const void* dens, void* Lexp, cudaStream_t s, int* launches);
int bem_run_m2p_t(bem_handle* h, int nrhs, const void* dens, void* Mu, cudaStream_t s, int* launches);
int bem_run_p2l_t(bem_handle* h, int nrhs, const void* Lam, double4* uv, cudaStream_t s, int* launches);
// off-surface evaluation through the tree (bem_eval_fmm.cu): the upward pass
// alone (P2M, M2M of h->dens into h->Mexp), then per point the far boxes'
// multipoles (bem_wx.cu) and the near leaves' elements (bem_apply.cu).
// mode: 0 value, 1 gradient, 2 value and gradient; acc is FP64 complex
// [nrhs][np][ncomp] in the walk's point order: the far pass writes it and
// flags the points with near leaves, the near pass (one warp per flagged
// point) adds to it, and bem_evf_out writes out[r][perm[i]][c] in the
// caller's dtype.  refine = 0 sums every near element with the regular
// 3-point rule R_0 (the vertex gradient's target side), 1 with the rule its
// distance calls for.
struct WalkTree;
int bem_run_upward(bem_handle* h, int nrhs, cudaStream_t s);
int bem_evf_far(bem_handle* h, const WalkTree& wt, int nrhs, int mode, int64_t np, const double* pts,
                const int* tcs, double* acc, int* nearflag, int team, cudaStream_t s);
int bem_evf_near(bem_handle* h, const WalkTree& wt, int nrhs, int mode, int64_t np, const double* pts,
                 const int* tcs, const int* near_list, const int* n_near, double* acc, int refine,
                 cudaStream_t s);
// The far pass of the vertex gradient's source side: the multipoles in h->Mexp
// are those of point charges at the centroids; at every walk point (a
// quadrature point of element perm[i] / 3, normal n) it writes FP64 complex
// acc[r][i][8] = (psi, grad psi, n.grad psi, (Hess psi) n) of the far boxes,
// the second derivatives by dual numbers along n.  team: lanes per point (a
// power of two up to 32) that share the point's far boxes; bem_evf_far takes
// the same (1 for the off-surface evaluation).
int bem_gvf_far(bem_handle* h, const WalkTree& wt, int nrhs, int64_t np, const double* pts, const int* tcs,
                const int* perm, int team, double* acc, cudaStream_t s);
int bem_evf_out(int nrhs, int mode, int64_t np, const int* perm, const double* acc, int dtype, void* out,
                cudaStream_t s);
int bem_eval_fmm(bem_handle* h, int nrhs, int dtype, const void* x, const void* y, const double* points,
                 int64_t np, void* out, int mode, cudaStream_t s);
int bem_build_correction(bem_handle* h, cudaStream_t s);
int bem_build_far_field(bem_handle* h, cudaStream_t s);
int bem_apply_sorted(bem_handle* h, int nrhs, cudaStream_t s);  // dens -> zn, zfar
int bem_apply_adjoint_sorted(bem_handle* h, int nrhs, cudaStream_t s);
int bem_prologue(bem_handle* h, int nrhs, int dtype, const void* x, const void* y, cudaStream_t s);
int bem_epilogue(bem_handle* h, int nrhs, int dtype, const void* x, void* z, int half, cudaStream_t s);
int bem_adjoint_prologue(bem_handle* h, int nrhs, int dtype, const void* g, cudaStream_t s);
int bem_adjoint_epilogue(bem_handle* h, int nrhs, int dtype, const void* g, void* gx, void* gy, int half,
                         cudaStream_t s);
// apply callback of the GMRES core: out = A in, both block vectors of complex FP64
typedef int (*bem_gm_apply_fn)(void* ctx, const double* in, double* out, cudaStream_t s);
// restarted GMRES on ncol independent systems in lockstep; column c is the
// segment [off[c], off[c] + len[c]) of a block vector of M complex entries.
// capture_apply (nullable) issues the same work as apply on the given stream
// with nothing that breaks stream capture (no synchronisation, allocation or
// events); with it the restart cycles run as CUDA graphs.
int bem_gmres_coupled(bem_handle* h, int nrhs, int dtype, const void* b_in, void* x_out, double tol, int max_iter,
                      int restart, bem_coupling_fn cb, void* cb_ctx, double* cx, double* cy, int flags,
                      int* iters_out, double* relres_out, cudaStream_t s);
int bem_gmres_core(bem_gm_apply_fn apply, bem_gm_apply_fn capture_apply, void* ctx, int ncol, int64_t M, const int64_t* off, const int64_t* len,
                   int dtype, const void* b, void* x, double tol, int max_iter, int restart, int flags,
                   int* iters_out, double* relres_out, cudaStream_t s);
int bem_gmres(bem_handle* h, int nrhs, int dtype, const void* b, void* x, double tol, int max_iter, int restart,
              int flags, int* iters_out, double* relres_out, cudaStream_t s);
int bem_check_device_error(bem_handle* h, cudaStream_t s);
int bem_build_tc(bem_handle* h, GroupedOp& op, int src_level, cudaStream_t s);
int bem_build_corr_transpose(bem_handle* h, cudaStream_t s);
int bem_build_adjoint(bem_handle* h, cudaStream_t s);
int bem_adjoint_sorted(bem_handle* h, int nrhs, int dtype, const void* g, void* gx, void* gy, int half,
                       cudaStream_t s);
int bem_run_grouped(bem_handle* h, GroupedOp& op, const void* src, void* dst, int nrhs, cudaStream_t s,
                    int* launches);
int bem_run_grouped_tc(bem_handle* h, GroupedOp& op, const void* src, void* dst, int nrhs, cudaStream_t s,
                       int* launches);
