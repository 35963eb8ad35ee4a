// bem_isosurface.cu -- the boundary Gamma = {phi = t} of the level-set region
// {phi > t} (Section 2.4: the elastic body is where phi > 0, the fluid where
// phi <= 0) as a closed triangle mesh, by marching tetrahedra on the grid.
//
// Every cube of the grid splits into the 6 tetrahedra that run from its
// corner (0,0,0) to (1,1,1) along the 6 orders of the axes.  The split is
// conforming: its edges run from a grid point g along one of 7 directions
// (three axes, three face diagonals, the body diagonal), so an edge is named
// (g, d) and a cut point is shared by every tetrahedron around its edge.
//
// Four passes, all one thread per grid point or cube (HBM-bound):
//   k_iso_mask    7-bit mask of the cut edges of every grid point and its count;
//   k_iso_count   triangles of every cube (1 per tetrahedron with 1 or 3
//                 corners inside, 2 with 2 inside);
//   two exclusive scans give vertex and triangle offsets, so the output order
//   is (g, d) for vertices and (cube, tetrahedron, piece) for triangles;
//   k_iso_vertices, k_iso_triangles write the mesh.
// The cut point of edge (a, b), a its lower end, is a + s (b - a) with
// s = (t - phi_a) / (phi_b - phi_a) clamped to [0.02, 0.98] (no degenerate
// triangles), in unfused IEEE operations.

#include <cub/cub.cuh>

#include <cstring>
#include <mutex>

#include "bem_common.cuh"

namespace {

__constant__ int c_dir[7][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};
// direction index of a 0/1 step vector, by its bits x | y << 1 | z << 2
__constant__ int c_dir_of_bits[8] = {-1, 0, 1, 3, 2, 4, 5, 6};
// the 6 axis orders of the split
__constant__ int c_perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

struct Grid {
  int n0, n1, n2;
  double lo0, lo1, lo2, h, t;
  long long tkey;  // order key of t
};

// An integer key of a double's bits that orders as the doubles do (NaN
// aside; -0 folds onto +0), so phi > t is decided on the integer pipe:
// FP64 instructions are slow on this part and cost a whole warp's issue
// even with one lane active.
__host__ __device__ __forceinline__ long long order_key(long long bits) {
  if (bits == (long long)0x8000000000000000ULL) bits = 0;
  return bits >= 0 ? bits : bits ^ 0x7FFFFFFFFFFFFFFFLL;
}
__device__ __forceinline__ bool above(const Grid& G, double f) { return order_key(__double_as_longlong(f)) > G.tkey; }

__device__ __forceinline__ int64_t gidx(const Grid& G, int i, int j, int k) {
  return ((int64_t)i * G.n1 + j) * G.n2 + k;
}

// corner c (0..3) of tetrahedron p as a 0/1 step from the cube's lower corner
__device__ __forceinline__ void corner(int p, int c, int v[3]) {
  v[0] = v[1] = v[2] = 0;
  for (int a = 0; a < c; ++a) v[c_perm[p][a]] = 1;
}

__global__ void k_iso_mask(Grid G, const double* __restrict__ phi, unsigned char* __restrict__ mask,
                           int* __restrict__ vcnt, int* __restrict__ bad) {
  const int64_t n = (int64_t)G.n0 * G.n1 * G.n2;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(g % G.n2), j = (int)((g / G.n2) % G.n1), i = (int)(g / ((int64_t)G.n1 * G.n2));
    const double f = phi[g];
    if (((__double_as_longlong(f) >> 52) & 0x7FF) == 0x7FF) atomicExch(bad, 1);  // NaN or infinity
    const bool in = above(G, f);
    unsigned m = 0;
#pragma unroll
    for (int d = 0; d < 7; ++d) {
      const int a = i + c_dir[d][0], b = j + c_dir[d][1], c = k + c_dir[d][2];
      if (a < G.n0 && b < G.n1 && c < G.n2 && above(G, phi[gidx(G, a, b, c)]) != in) m |= 1u << d;
    }
    mask[g] = (unsigned char)m;
    vcnt[g] = __popc(m);
  }
}

__global__ void k_iso_count(Grid G, const double* __restrict__ phi, int* __restrict__ tcnt) {
  const int c1 = G.n1 - 1, c2 = G.n2 - 1;
  const int64_t n = (int64_t)(G.n0 - 1) * c1 * c2;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(c % c2), j = (int)((c / c2) % c1), i = (int)(c / ((int64_t)c1 * c2));
    unsigned in8 = 0;  // bit x | y << 1 | z << 2: the cube corner at that step is inside
    for (int b = 0; b < 8; ++b)
      if (above(G, phi[gidx(G, i + (b & 1), j + ((b >> 1) & 1), k + (b >> 2))])) in8 |= 1u << b;
    int tot = 0;
    if (in8 != 0 && in8 != 255)
      for (int p = 0; p < 6; ++p) {
        int nin = 0;
        for (int q = 0; q < 4; ++q) {
          int v[3];
          corner(p, q, v);
          nin += (in8 >> (v[0] | v[1] << 1 | v[2] << 2)) & 1;
        }
        tot += (nin == 1 || nin == 3) ? 1 : (nin == 2 ? 2 : 0);
      }
    tcnt[c] = tot;
  }
}

__global__ void k_iso_vertices(Grid G, const double* __restrict__ phi, const unsigned char* __restrict__ mask,
                               const int* __restrict__ vbase, double* __restrict__ V) {
  const int64_t n = (int64_t)G.n0 * G.n1 * G.n2;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const unsigned m = mask[g];
    if (!m) continue;
    const int k = (int)(g % G.n2), j = (int)((g / G.n2) % G.n1), i = (int)(g / ((int64_t)G.n1 * G.n2));
    const double fa = phi[g];
    const double pa[3] = {__dadd_rn(G.lo0, __dmul_rn((double)i, G.h)), __dadd_rn(G.lo1, __dmul_rn((double)j, G.h)),
                          __dadd_rn(G.lo2, __dmul_rn((double)k, G.h))};
    int v = vbase[g];
    for (int d = 0; d < 7; ++d) {
      if (!((m >> d) & 1)) continue;
      const int ib = i + c_dir[d][0], jb = j + c_dir[d][1], kb = k + c_dir[d][2];
      const double fb = phi[gidx(G, ib, jb, kb)];
      double s = __ddiv_rn(__dsub_rn(G.t, fa), __dsub_rn(fb, fa));
      s = fmin(fmax(s, 0.02), 0.98);
      const double pb[3] = {__dadd_rn(G.lo0, __dmul_rn((double)ib, G.h)),
                            __dadd_rn(G.lo1, __dmul_rn((double)jb, G.h)),
                            __dadd_rn(G.lo2, __dmul_rn((double)kb, G.h))};
      for (int a = 0; a < 3; ++a) V[3 * (int64_t)v + a] = __dadd_rn(pa[a], __dmul_rn(s, __dsub_rn(pb[a], pa[a])));
      ++v;
    }
  }
}

// vertex id of the cut edge between cube corners with steps u < w (componentwise)
__device__ __forceinline__ int edge_vertex(const Grid& G, const unsigned char* mask, const int* vbase, int i, int j,
                                           int k, const int u[3], const int w[3]) {
  const int d = c_dir_of_bits[(w[0] - u[0]) | (w[1] - u[1]) << 1 | (w[2] - u[2]) << 2];
  const int64_t g = gidx(G, i + u[0], j + u[1], k + u[2]);
  return vbase[g] + __popc(mask[g] & ((1u << d) - 1));
}

__global__ void k_iso_triangles(Grid G, const double* __restrict__ phi, const unsigned char* __restrict__ mask,
                                const int* __restrict__ vbase, const int* __restrict__ tcnt,
                                const int* __restrict__ tbase, const double* __restrict__ V, int* __restrict__ T) {
  const int c1 = G.n1 - 1, c2 = G.n2 - 1;
  const int64_t n = (int64_t)(G.n0 - 1) * c1 * c2;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    if (tcnt[c] == 0) continue;
    const int k = (int)(c % c2), j = (int)((c / c2) % c1), i = (int)(c / ((int64_t)c1 * c2));
    int out = tbase[c];
    for (int p = 0; p < 6; ++p) {
      int cv[4][3];
      bool in[4];
      int nin = 0;
      for (int q = 0; q < 4; ++q) {
        corner(p, q, cv[q]);
        in[q] = above(G, phi[gidx(G, i + cv[q][0], j + cv[q][1], k + cv[q][2])]);
        nin += in[q];
      }
      if (nin == 0 || nin == 4) continue;
      int ins[3], outs[3], ni = 0, no = 0;
      for (int q = 0; q < 4; ++q) {
        if (in[q]) ins[ni++] = q;
        else outs[no++] = q;
      }
      // corners are numbered along the path (0,0,0) -> (1,1,1), so q < r means step q <= step r
#define ISO_CUT(qa, qb) \
  ((qa) < (qb) ? edge_vertex(G, mask, vbase, i, j, k, cv[qa], cv[qb]) : edge_vertex(G, mask, vbase, i, j, k, cv[qb], cv[qa]))
      int tri[2][3], ntri;
      if (nin == 1 || nin == 3) {
        const int lone = nin == 1 ? ins[0] : outs[0];
        const int* rest = nin == 1 ? outs : ins;
        for (int a = 0; a < 3; ++a) tri[0][a] = ISO_CUT(lone, rest[a]);
        ntri = 1;
      } else {
        const int q0 = ISO_CUT(ins[0], outs[0]), q1 = ISO_CUT(ins[0], outs[1]), q2 = ISO_CUT(ins[1], outs[1]),
                  q3 = ISO_CUT(ins[1], outs[0]);
        tri[0][0] = q0, tri[0][1] = q1, tri[0][2] = q2;
        tri[1][0] = q0, tri[1][1] = q2, tri[1][2] = q3;
        ntri = 2;
      }
#undef ISO_CUT
      // face from the inside corners to the outside ones: the cut plane
      // separates them, so the sign of this test is never close to zero.
      // away = nin (4 - nin) (mean of the outside corners - mean of the
      // inside ones), in integers: the positive factor keeps the sign.
      int awi[3] = {0, 0, 0};
      for (int q = 0; q < 4; ++q)
        for (int a = 0; a < 3; ++a) awi[a] += in[q] ? -(4 - nin) * cv[q][a] : nin * cv[q][a];
      const double away[3] = {(double)awi[0], (double)awi[1], (double)awi[2]};
      for (int s = 0; s < ntri; ++s) {
        const double* A = V + 3 * (int64_t)tri[s][0];
        const double* B = V + 3 * (int64_t)tri[s][1];
        const double* C = V + 3 * (int64_t)tri[s][2];
        const double e1[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]}, e2[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
        const double nr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        const bool flip = nr[0] * away[0] + nr[1] * away[1] + nr[2] * away[2] < 0.0;
        T[3 * (int64_t)out] = tri[s][0];
        T[3 * (int64_t)out + 1] = flip ? tri[s][2] : tri[s][1];
        T[3 * (int64_t)out + 2] = flip ? tri[s][1] : tri[s][2];
        ++out;
      }
    }
  }
}

__global__ void k_iso_totals(int64_t npt, int64_t ncube, const int* vbase, const int* vcnt, const int* tbase,
                             const int* tcnt, const int* bad, int* tot) {
  tot[0] = vbase[npt - 1] + vcnt[npt - 1];
  tot[1] = tbase[ncube - 1] + tcnt[ncube - 1];
  tot[2] = *bad;
}

unsigned iso_blocks(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 64));
}

// Grow-only scratch, one per process, reused by later calls (a call
// synchronises its stream before it returns, so calls hold the lock for their
// whole duration and never share buffers in flight).
struct IsoScratch {
  std::mutex mu;
  int device = -1;
  int64_t npt = 0, ncube = 0;
  size_t tmp_bytes = 0;
  unsigned char* mask = nullptr;
  int *vcnt = nullptr, *vbase = nullptr, *tcnt = nullptr, *tbase = nullptr, *flags = nullptr;
  void* tmp = nullptr;

  void release() {
    cudaFree(mask), cudaFree(vcnt), cudaFree(vbase), cudaFree(tcnt), cudaFree(tbase), cudaFree(flags), cudaFree(tmp);
    mask = nullptr, vcnt = vbase = tcnt = tbase = flags = nullptr, tmp = nullptr;
    npt = ncube = 0, tmp_bytes = 0;
  }
  cudaError_t reserve(int dev, int64_t np, int64_t nc, size_t tb) {
    if (dev == device && np <= npt && nc <= ncube && tb <= tmp_bytes) return cudaSuccess;
    if (dev != device) release();
    np = std::max(np, npt), nc = std::max(nc, ncube), tb = std::max(tb, tmp_bytes);
    release();
    cudaError_t e;
    if ((e = cudaMalloc((void**)&mask, np)) != cudaSuccess) return e;
    if ((e = cudaMalloc((void**)&vcnt, np * sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMalloc((void**)&vbase, np * sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMalloc((void**)&tcnt, nc * sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMalloc((void**)&tbase, nc * sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMalloc((void**)&flags, 4 * sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&tmp, tb)) != cudaSuccess) return e;
    device = dev, npt = np, ncube = nc, tmp_bytes = tb;
    return cudaSuccess;
  }
};
IsoScratch g_iso;

}  // namespace

int bem_isosurface(int n0, int n1, int n2, const double* phi, const double* lo, double h, double t, double* vertices,
                   int64_t max_vertices, int* triangles, int64_t max_triangles, int64_t* counts, void* stream) {
  bem_set_error("");
  if (!phi || !lo || !counts) return bem_fail(BEM_ERR_INVALID_ARG, "phi, lo or counts is NULL");
  if (n0 < 2 || n1 < 2 || n2 < 2) return bem_fail(BEM_ERR_INVALID_ARG, "the grid needs at least 2 points per axis");
  if (!(h > 0.0) || !std::isfinite(h) || !std::isfinite(t) || !std::isfinite(lo[0]) || !std::isfinite(lo[1]) ||
      !std::isfinite(lo[2]))
    return bem_fail(BEM_ERR_INVALID_ARG, "h must be positive; lo and t finite");
  const int64_t npt = (int64_t)n0 * n1 * n2, ncube = (int64_t)(n0 - 1) * (n1 - 1) * (n2 - 1);
  // offsets are int32: 7 vertices per grid point and 12 triangles per cube at most
  if (7 * npt >= INT32_MAX || 12 * ncube >= INT32_MAX)
    return bem_fail(BEM_ERR_INVALID_ARG, "grid too large for 32-bit vertex and triangle indices");
  cudaStream_t s = (cudaStream_t)stream;
  long long tbits;
  std::memcpy(&tbits, &t, sizeof(tbits));
  const Grid G{n0, n1, n2, lo[0], lo[1], lo[2], h, t, order_key(tbits)};
  size_t tb1 = 0, tb2 = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, tb1, (int*)nullptr, (int*)nullptr, (int)npt, s);
  cub::DeviceScan::ExclusiveSum(nullptr, tb2, (int*)nullptr, (int*)nullptr, (int)ncube, s);
  int dev = 0;
  BEM_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_iso.mu);
  {
    const cudaError_t e = g_iso.reserve(dev, npt, ncube, std::max(tb1, tb2) + 16);
    if (e != cudaSuccess) {
      g_iso.release();
      cudaGetLastError();
      return bem_fail(e == cudaErrorMemoryAllocation ? BEM_ERR_OOM : BEM_ERR_CUDA, cudaGetErrorString(e));
    }
  }
  IsoScratch& W = g_iso;
  int* tot = W.flags + 1;  // device: vertex count, triangle count, bad flag
  int host[3] = {0, 0, 0};
  BEM_CUDA(cudaMemsetAsync(W.flags, 0, sizeof(int), s));
  k_iso_mask<<<iso_blocks(npt), 256, 0, s>>>(G, phi, W.mask, W.vcnt, W.flags);
  k_iso_count<<<iso_blocks(ncube), 256, 0, s>>>(G, phi, W.tcnt);
  BEM_CUDA(cudaGetLastError());
  BEM_CUDA(cub::DeviceScan::ExclusiveSum(W.tmp, tb1, W.vcnt, W.vbase, (int)npt, s));
  BEM_CUDA(cub::DeviceScan::ExclusiveSum(W.tmp, tb2, W.tcnt, W.tbase, (int)ncube, s));
  k_iso_totals<<<1, 1, 0, s>>>(npt, ncube, W.vbase, W.vcnt, W.tbase, W.tcnt, W.flags, tot);
  BEM_CUDA(cudaGetLastError());
  BEM_CUDA(cudaMemcpyAsync(host, tot, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
  BEM_CUDA(cudaStreamSynchronize(s));
  counts[0] = host[0];
  counts[1] = host[1];
  if (host[2]) return bem_fail(BEM_ERR_NUMERIC, "phi holds a NaN or an infinity");
  if (vertices && triangles) {
    if (counts[0] > max_vertices || counts[1] > max_triangles)
      return bem_fail(BEM_ERR_INVALID_ARG, "vertex or triangle capacity below the counts (counts filled)");
    k_iso_vertices<<<iso_blocks(npt), 256, 0, s>>>(G, phi, W.mask, W.vbase, vertices);
    k_iso_triangles<<<iso_blocks(ncube), 256, 0, s>>>(G, phi, W.mask, W.vbase, W.tcnt, W.tbase, vertices, triangles);
    BEM_CUDA(cudaGetLastError());
    // the scratch is reused by the next call: finish before the lock is released
    BEM_CUDA(cudaStreamSynchronize(s));
  }
  return BEM_OK;
}
