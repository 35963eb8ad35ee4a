// bem_eval_fmm.cu -- the field (and its gradient) at points off the surface
// through the FMM (Section 2.3's tree evaluating the representation formula
// at field points, as the topological derivative of Section 2.5 needs on a
// lattice):
//   1. prologue: the weighted densities in tree order;
//   2. upward pass: P2M of every leaf, M2M up to level 2;
//   3. the points are sorted along a Morton curve of their level-L boxes
//      (extended beyond the root cube), so that the threads of a warp walk
//      nearly the same boxes;
//   4. far pass: per point, the multipole of every far box of its walk;
//   5. near pass: one warp per point whose walk has near leaves (flagged by
//      the far pass, compacted), the lanes splitting the leaves' elements;
//   6. the FP64 sums written in the caller's point order and dtype.
// Temporary arrays are stream-ordered allocations freed at the end of the call.
#include <cub/cub.cuh>

#include "bem_common.cuh"
#include "bem_tree_walk.cuh"

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

WalkTree bem_walk_tree(const bem_handle* h) {
  WalkTree wt;
  wt.L = h->L;
  for (int d = 0; d < 3; ++d) wt.lo[d] = h->root_c[d] - 0.5 * h->root_w;
  wt.wL = h->root_w / (double)(1 << h->L);
  for (int l = 0; l <= h->L; ++l) {
    const LevelInfo& lv = h->lev[l];
    WalkLevel& w = wt.lv[l];
    w.coord = lv.coord;
    w.internal = lv.internal;
    w.child0 = lv.child0;
    w.nchild = lv.nchild;
    w.gap2 = lv.gap2;
    w.centre = lv.centre;
    w.start = lv.start;
    w.end = lv.end;
    w.nbox = lv.nbox;
  }
  return wt;
}

// spread the low 21 bits of v to every third bit
__device__ __forceinline__ unsigned long long spread3(unsigned long long v) {
  v &= 0x1FFFFFULL;
  v = (v | (v << 32)) & 0x1F00000000FFFFULL;
  v = (v | (v << 16)) & 0x1F0000FF0000FFULL;
  v = (v | (v << 8)) & 0x100F00F00F00F00FULL;
  v = (v | (v << 4)) & 0x10C30C30C30C30C3ULL;
  v = (v | (v << 2)) & 0x1249249249249249ULL;
  return v;
}

__global__ void k_evf_keys(int64_t np, WalkTree wt, const double* __restrict__ pts, unsigned long long* keys,
                           int* idx) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  int t[3];
  walk_box_of(wt, pts + 3 * i, t);
  // coordinates in [-2^20, 2^20 - 1], shifted to [0, 2^21 - 1]
  keys[i] = (spread3((unsigned long long)(t[0] + WALK_COORD_MAX)) << 2) |
            (spread3((unsigned long long)(t[1] + WALK_COORD_MAX)) << 1) |
            spread3((unsigned long long)(t[2] + WALK_COORD_MAX));
  idx[i] = (int)i;
}

__global__ void k_evf_gather(int64_t np, WalkTree wt, const int* __restrict__ perm, const double* __restrict__ pts,
                             double* __restrict__ spts, int* __restrict__ tcs) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int64_t o = perm[i];
  const double X[3] = {pts[3 * o], pts[3 * o + 1], pts[3 * o + 2]};
  int t[3];
  walk_box_of(wt, X, t);
  for (int a = 0; a < 3; ++a) {
    spts[3 * i + a] = X[a];
    tcs[3 * i + a] = t[a];
  }
}

static int walk_fail(cudaError_t e) {
  return bem_fail(e == cudaErrorMemoryAllocation ? BEM_ERR_OOM : BEM_ERR_CUDA, cudaGetErrorString(e));
}
#define WALK_CUDA(call)                      \
  do {                                       \
    const cudaError_t e_ = (call);           \
    if (e_ != cudaSuccess) return walk_fail(e_); \
  } while (0)

int bem_walk_order(const WalkTree& wt, int64_t np, const double* points, WalkOrder& wo, cudaStream_t s) {
  if (np > 0x7fffffffLL) return bem_fail(BEM_ERR_INVALID_ARG, "too many points for one call");
  WALK_CUDA(cudaMallocAsync((void**)&wo.keys_in, np * sizeof(unsigned long long), s));
  WALK_CUDA(cudaMallocAsync((void**)&wo.keys, np * sizeof(unsigned long long), s));
  WALK_CUDA(cudaMallocAsync((void**)&wo.idx_in, np * sizeof(int), s));
  WALK_CUDA(cudaMallocAsync((void**)&wo.perm, np * sizeof(int), s));
  WALK_CUDA(cudaMallocAsync((void**)&wo.tcs, 3 * np * sizeof(int), s));
  WALK_CUDA(cudaMallocAsync((void**)&wo.spts, 3 * np * sizeof(double), s));
  WALK_CUDA(cudaMallocAsync((void**)&wo.nearflag, np * sizeof(int), s));
  WALK_CUDA(cudaMallocAsync((void**)&wo.near_list, np * sizeof(int), s));
  WALK_CUDA(cudaMallocAsync((void**)&wo.n_near, sizeof(int), s));
  k_evf_keys<<<nblk(np, 256), 256, 0, s>>>(np, wt, points, wo.keys_in, wo.idx_in);
  WALK_CUDA(cudaGetLastError());
  size_t tb = 0;
  WALK_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tb, wo.keys_in, wo.keys, wo.idx_in, wo.perm, (int)np, 0, 63, s));
  WALK_CUDA(cudaMallocAsync(&wo.tmp, tb, s));
  WALK_CUDA(cub::DeviceRadixSort::SortPairs(wo.tmp, tb, wo.keys_in, wo.keys, wo.idx_in, wo.perm, (int)np, 0, 63, s));
  k_evf_gather<<<nblk(np, 256), 256, 0, s>>>(np, wt, wo.perm, points, wo.spts, wo.tcs);
  WALK_CUDA(cudaGetLastError());
  return BEM_OK;
}

int bem_walk_near_list(int64_t np, WalkOrder& wo, cudaStream_t s) {
  // the points whose walk has near leaves, in walk order (idx_in still holds
  // 0 .. np - 1: the sort wrote its output to perm)
  size_t tb2 = 0;
  WALK_CUDA(cub::DeviceSelect::Flagged(nullptr, tb2, wo.idx_in, wo.nearflag, wo.near_list, wo.n_near, (int)np, s));
  WALK_CUDA(cudaMallocAsync(&wo.tmp2, tb2, s));
  WALK_CUDA(cub::DeviceSelect::Flagged(wo.tmp2, tb2, wo.idx_in, wo.nearflag, wo.near_list, wo.n_near, (int)np, s));
  return BEM_OK;
}

void bem_walk_free(WalkOrder& wo, cudaStream_t s) {
  for (void* p : {(void*)wo.keys_in, (void*)wo.keys, (void*)wo.idx_in, (void*)wo.perm, (void*)wo.tcs,
                  (void*)wo.spts, (void*)wo.nearflag, (void*)wo.near_list, (void*)wo.n_near, wo.tmp, wo.tmp2})
    if (p) cudaFreeAsync(p, s);
  wo = WalkOrder();
}

int bem_eval_fmm(bem_handle* h, int nrhs, int dtype, const void* x, const void* y, const double* points,
                 int64_t np, void* out, int mode, cudaStream_t s) {
  if (np > 0x7fffffffLL) return bem_fail(BEM_ERR_INVALID_ARG, "too many points for one call");
  const WalkTree wt = bem_walk_tree(h);
  const int nc = mode == 0 ? 1 : (mode == 1 ? 3 : 4);
  BEM_TRY(bem_prologue(h, nrhs, dtype, x, y, s));
  BEM_TRY(bem_run_upward(h, nrhs, s));
  WalkOrder wo;
  double* acc = nullptr;
  int rc = BEM_OK;
  do {
    const cudaError_t e = cudaMallocAsync((void**)&acc, 2 * nc * nrhs * np * sizeof(double), s);
    if (e != cudaSuccess) {
      rc = walk_fail(e);
      break;
    }
    if ((rc = bem_walk_order(wt, np, points, wo, s)) != BEM_OK) break;
    if ((rc = bem_evf_far(h, wt, nrhs, mode, np, wo.spts, wo.tcs, acc, wo.nearflag, 1, s)) != BEM_OK) break;
    if ((rc = bem_walk_near_list(np, wo, s)) != BEM_OK) break;
    if ((rc = bem_evf_near(h, wt, nrhs, mode, np, wo.spts, wo.tcs, wo.near_list, wo.n_near, acc, 1, s)) != BEM_OK)
      break;
    rc = bem_evf_out(nrhs, mode, np, wo.perm, acc, dtype, out, s);
  } while (false);
  if (acc) cudaFreeAsync(acc, s);
  bem_walk_free(wo, s);
  return rc;
}
