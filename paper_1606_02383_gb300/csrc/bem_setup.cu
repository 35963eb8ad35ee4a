// bem_setup.cu -- geometry, octree, interaction lists and the FP64 near-singular
// correction matrix.
//
// Geometry (Section 2.3: flat triangles, piecewise-constant densities,
// collocation at centroids): centroid c_j, area A_j, unit normal n_j
// ((b-a)x(c-a) normalised, pointing into the fluid, Section 2.1), longest edge
// h_j, and the three points of the regular rule (barycentric (2/3,1/6,1/6) and
// permutations, weight A_j/3 each).
//
// Octree: 30-bit Morton keys (10 bits per axis) of the centroids in the root
// cube, sorted with CUB's radix sort; level-l boxes are the distinct key
// prefixes, so every box owns a contiguous range of sorted elements.  Lists:
// the 27 colleagues of every leaf (near field) and, on every level >= 2, the
// V-list (children of the parent's colleagues that are not adjacent), grouped
// by the offset between the two boxes so that each group shares one
// translation matrix.
//
// Near-singular correction: for every target i and source j != i with
// |x_i - c_j| < 4 h_j, C_ij = (entry by the refined rule R_L) - (entry by the
// regular rule R_0), and C_ii = the exact self term, for S and D, in FP64.
// The apply evaluates R_0 for every other pair (near field directly, far
// field by the FMM) and adds C, which reproduces the rule-defined operator;
// the self pair never passes through the FP32 near field, so its D_ii = 0
// and S_ii keep FP64 accuracy whatever the size of the leaf box.
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "bem_common.cuh"
#include "bem_rules.cuh"

// ----------------------------------------------------------------- helpers --
__device__ __forceinline__ void dev_flag(int* err, int bit) { atomicOr(err, bit); }

__device__ __forceinline__ uint32_t spread3(uint32_t v) {  // 10 bits -> every third bit
  v &= 0x3ff;
  v = (v | (v << 16)) & 0x030000FF;
  v = (v | (v << 8)) & 0x0300F00F;
  v = (v | (v << 4)) & 0x030C30C3;
  v = (v | (v << 2)) & 0x09249249;
  return v;
}
__device__ __forceinline__ uint32_t compact3(uint32_t v) {
  v &= 0x09249249;
  v = (v ^ (v >> 2)) & 0x030C30C3;
  v = (v ^ (v >> 4)) & 0x0300F00F;
  v = (v ^ (v >> 8)) & 0x030000FF;
  v = (v ^ (v >> 16)) & 0x000003FF;
  return v;
}
__device__ __forceinline__ uint32_t morton3(uint32_t x, uint32_t y, uint32_t z) {
  return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

// ----------------------------------------------------------------- geometry --
// Per triangle in the caller's order.
__global__ void k_geometry(const double* __restrict__ V, const int32_t* __restrict__ T, int64_t nt, int64_t nv,
                           double* cent, double* qpt, double* nrm, double* area, double* hmax, int* err) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= nt) return;
  double v[3][3];
  for (int a = 0; a < 3; ++a) {
    int32_t id = T[3 * j + a];
    if (id < 0 || id >= nv) {
      dev_flag(err, BEM_DEVERR_DEGENERATE);
      id = 0;
    }
    for (int d = 0; d < 3; ++d) v[a][d] = V[3 * (int64_t)id + d];
  }
  double e1[3], e2[3], e3[3];
  for (int d = 0; d < 3; ++d) {
    e1[d] = v[1][d] - v[0][d];
    e2[d] = v[2][d] - v[0][d];
    e3[d] = v[2][d] - v[1][d];
  }
  double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
  double len = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
  double h1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
  double h2 = sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]);
  double h3 = sqrt(e3[0] * e3[0] + e3[1] * e3[1] + e3[2] * e3[2]);
  double h = fmax(h1, fmax(h2, h3));
  if (!(len > 1e-300) || !isfinite(len) || !(len > 1e-14 * h * h)) {
    dev_flag(err, BEM_DEVERR_DEGENERATE);
    len = 1.0;
  }
  area[j] = 0.5 * len;
  hmax[j] = h;
  for (int d = 0; d < 3; ++d) {
    nrm[3 * j + d] = cr[d] / len;
    cent[3 * j + d] = (v[0][d] + v[1][d] + v[2][d]) / 3.0;
  }
  const double b0 = 2.0 / 3.0, b1 = 1.0 / 6.0;
  for (int q = 0; q < 3; ++q)
    for (int d = 0; d < 3; ++d)
      qpt[9 * j + 3 * q + d] = (q == 0 ? b0 : b1) * v[0][d] + (q == 1 ? b0 : b1) * v[1][d] + (q == 2 ? b0 : b1) * v[2][d];
}

// block-wise min/max of the vertex coordinates
__global__ void k_bbox(const double* __restrict__ V, int64_t nv, double* out) {
  __shared__ double sm[6][256];
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x)
    for (int d = 0; d < 3; ++d) {
      double x = V[3 * i + d];
      lo[d] = fmin(lo[d], x);
      hi[d] = fmax(hi[d], x);
    }
  for (int d = 0; d < 3; ++d) {
    sm[d][threadIdx.x] = lo[d];
    sm[3 + d][threadIdx.x] = hi[d];
  }
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int d = 0; d < 3; ++d) {
        sm[d][threadIdx.x] = fmin(sm[d][threadIdx.x], sm[d][threadIdx.x + s]);
        sm[3 + d][threadIdx.x] = fmax(sm[3 + d][threadIdx.x], sm[3 + d][threadIdx.x + s]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int d = 0; d < 6; ++d) out[6 * blockIdx.x + d] = sm[d][0];
}

__global__ void k_morton(const double* __restrict__ cent, int64_t nt, double lo0, double lo1, double lo2, double wfine,
                         uint32_t* keys, int* idx) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= nt) return;
  uint32_t c[3];
  double lo[3] = {lo0, lo1, lo2};
  for (int d = 0; d < 3; ++d) {
    double f = floor((cent[3 * j + d] - lo[d]) / wfine);
    f = fmin(fmax(f, 0.0), 1023.0);
    c[d] = (uint32_t)f;
  }
  keys[j] = morton3(c[0], c[1], c[2]);
  idx[j] = (int)j;
}

// number of distinct prefixes at every level (sorted keys)
__global__ void k_count_levels(const uint32_t* __restrict__ keys, int64_t nt, unsigned long long* counts) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nt) return;
  for (int l = 0; l <= BEM_MAXLEV; ++l) {
    int sh = 3 * (BEM_MAXLEV - l);
    bool first = (i == 0) || ((keys[i] >> sh) != (keys[i - 1] >> sh));
    if (first) atomicAdd(&counts[l], 1ull);
  }
}

// gather per-element geometry into sorted order
__global__ void k_permute_geometry(const int* __restrict__ perm, int64_t nt, const double* cent_o, const double* qpt_o,
                                   const double* nrm_o, const double* area_o, const double* hmax_o,
                                   const int32_t* __restrict__ tri_o, double* cent, double* qpt, double* nrm,
                                   double* area, double* hmax, double* wgt, int* tri) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nt) return;
  int64_t o = perm[s];
  for (int a = 0; a < 3; ++a) tri[3 * s + a] = tri_o[3 * o + a];
  for (int d = 0; d < 3; ++d) {
    cent[3 * s + d] = cent_o[3 * o + d];
    nrm[3 * s + d] = nrm_o[3 * o + d];
  }
  for (int d = 0; d < 9; ++d) qpt[9 * s + d] = qpt_o[9 * o + d];
  area[s] = area_o[o];
  hmax[s] = hmax_o[o];
  wgt[s] = area_o[o] / (12.0 * BEM_PI);
}

// box boundaries at one level: flags then scan
__global__ void k_level_flags(const uint32_t* __restrict__ keys, int64_t nt, int sh, int* flags) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nt) return;
  flags[i] = (i == 0 || (keys[i] >> sh) != (keys[i - 1] >> sh)) ? 1 : 0;
}

// elbox = inclusive scan - 1; write box start/key/coords/centre
__global__ void k_level_boxes(const uint32_t* __restrict__ keys, const int* __restrict__ scan, int64_t nt, int sh,
                              int l, double lo0, double lo1, double lo2, double w, int* elbox, uint32_t* bkey,
                              int* bstart, int* bend, int* coord, double* centre) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nt) return;
  int b = scan[i] - 1;
  elbox[i] = b;
  bool first = (i == 0 || (keys[i] >> sh) != (keys[i - 1] >> sh));
  bool last = (i == nt - 1 || (keys[i] >> sh) != (keys[i + 1] >> sh));
  if (first) {
    uint32_t pre = keys[i] >> sh;
    bkey[b] = pre;
    bstart[b] = (int)i;
    uint32_t cx = compact3(pre), cy = compact3(pre >> 1), cz = compact3(pre >> 2);
    coord[3 * b + 0] = (int)cx;
    coord[3 * b + 1] = (int)cy;
    coord[3 * b + 2] = (int)cz;
    centre[3 * b + 0] = lo0 + (cx + 0.5) * w;
    centre[3 * b + 1] = lo1 + (cy + 0.5) * w;
    centre[3 * b + 2] = lo2 + (cz + 0.5) * w;
  }
  if (last) bend[b] = (int)(i + 1);
  (void)l;
}

__global__ void k_level_links(int nbox, const int* __restrict__ bstart, const int* __restrict__ bend,
                              const int* __restrict__ elbox_up, const int* __restrict__ elbox_down, int* parent,
                              int* child0, int* nchild) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  parent[b] = elbox_up ? elbox_up[bstart[b]] : -1;
  if (elbox_down) {
    int c0 = elbox_down[bstart[b]];
    child0[b] = c0;
    nchild[b] = elbox_down[bend[b] - 1] - c0 + 1;
  } else {
    child0[b] = -1;
    nchild[b] = 0;
  }
}

// find the box with the given coordinates at a level (sorted keys); -1 if absent
__device__ __forceinline__ int find_box(const uint32_t* __restrict__ bkey, int nbox, int x, int y, int z, int side) {
  if (x < 0 || y < 0 || z < 0 || x >= side || y >= side || z >= side) return -1;
  uint32_t key = morton3((uint32_t)x, (uint32_t)y, (uint32_t)z);
  int lo = 0, hi = nbox - 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    uint32_t km = bkey[mid];
    if (km == key) return mid;
    if (km < key)
      lo = mid + 1;
    else
      hi = mid - 1;
  }
  return -1;
}

__global__ void k_colleagues(int nbox, const uint32_t* __restrict__ bkey, const int* __restrict__ coord, int side,
                             int* coll27) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  int cx = coord[3 * b], cy = coord[3 * b + 1], cz = coord[3 * b + 2];
  int t = 0;
  for (int dx = -1; dx <= 1; ++dx)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dz = -1; dz <= 1; ++dz) coll27[27 * b + (t++)] = find_box(bkey, nbox, cx + dx, cy + dy, cz + dz, side);
}

__global__ void k_count_p2p(int nleaf, const int* __restrict__ coll27, const int* __restrict__ bstart,
                            const int* __restrict__ bend, unsigned long long* pairs) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nleaf) return;
  long long ns = 0;
  for (int t = 0; t < 27; ++t) {
    int c = coll27[27 * b + t];
    if (c >= 0) ns += bend[c] - bstart[c];
  }
  atomicAdd(pairs, (unsigned long long)(ns * (bend[b] - bstart[b])));
}

// V-list of tree box b: children of the parent's internal colleagues that are
// not adjacent to b (a leaf colleague has no children in the tree; its
// elements reach b through the X-lists or the near field).  pass 0 counts per
// offset, pass 1 fills.
__global__ void k_vlist(int nbox, const int* __restrict__ coord, const int* __restrict__ parent,
                        const int* __restrict__ pcoll27, const int* __restrict__ pchild0,
                        const int* __restrict__ pnchild, const int* __restrict__ ccoord,
                        const unsigned char* __restrict__ intree, const unsigned char* __restrict__ pinternal, int pass,
                        int* counts, int* cursor, const int* __restrict__ gstart, int* src_box, int* dst_box) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  if (!intree[b]) return;
  int p = parent[b];
  int bx = coord[3 * b], by = coord[3 * b + 1], bz = coord[3 * b + 2];
  for (int t = 0; t < 27; ++t) {
    int q = pcoll27[27 * p + t];
    if (q < 0 || !pinternal[q]) continue;
    int c0 = pchild0[q], nc = pnchild[q];
    for (int c = c0; c < c0 + nc; ++c) {
      int dx = bx - ccoord[3 * c], dy = by - ccoord[3 * c + 1], dz = bz - ccoord[3 * c + 2];
      if (abs(dx) <= 1 && abs(dy) <= 1 && abs(dz) <= 1) continue;
      int o = (dx + 3) * 49 + (dy + 3) * 7 + (dz + 3);
      if (pass == 0) {
        atomicAdd(&counts[o], 1);
      } else {
        int pos = gstart[o] + atomicAdd(&cursor[o], 1);
        src_box[pos] = c;
        dst_box[pos] = b;
      }
    }
  }
}

// longest edge of every box (one block per box)
__global__ void k_box_hmax(int nbox, const int* __restrict__ bstart, const int* __restrict__ bend,
                           const double* __restrict__ hmax, double* out) {
  __shared__ double sm[128];
  const int b = blockIdx.x;
  double m = 0.0;
  for (int i = bstart[b] + threadIdx.x; i < bend[b]; i += blockDim.x) m = fmax(m, hmax[i]);
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[b] = sm[0];
}

// leaf membership of the elements of one level's leaves (one block per leaf)
__global__ void k_leaf_mark(int nleaf, const int* __restrict__ leafbox, const int* __restrict__ bstart,
                            const int* __restrict__ bend, int level, int g0, int* leaf_of, unsigned char* leaf_lev,
                            int* gleaf_of) {
  const int i = blockIdx.x;
  if (i >= nleaf) return;
  const int b = leafbox[i];
  for (int e = bstart[b] + threadIdx.x; e < bend[b]; e += blockDim.x) {
    leaf_of[e] = b;
    leaf_lev[e] = (unsigned char)level;
    gleaf_of[e] = g0 + i;
  }
}

// Exact self term S_ii: polar coordinates about the centroid, one sub-triangle per
// edge; with tan(phi) = sinh(u) the radial integral of exp(ik rho)/rho * rho is
// (exp(ik rho) - 1)/(ik) at rho = d cosh(u), and dphi = du / cosh(u).
__constant__ double c_gl_x[32];
__constant__ double c_gl_w[32];

__device__ zd self_single_layer(const Tri64& t, double k) {
  zd acc = cmk(0.0, 0.0);
  for (int e = 0; e < 3; ++e) {
    const double* a = t.v[e];
    const double* b = t.v[(e + 1) % 3];
    double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double len = sqrt(ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2]);
    double tv[3] = {ab[0] / len, ab[1] / len, ab[2] / len};
    double xa[3] = {t.c[0] - a[0], t.c[1] - a[1], t.c[2] - a[2]};
    double pr = xa[0] * tv[0] + xa[1] * tv[1] + xa[2] * tv[2];
    double fx[3] = {xa[0] - pr * tv[0], xa[1] - pr * tv[1], xa[2] - pr * tv[2]};  // centroid - foot
    double dist = sqrt(fx[0] * fx[0] + fx[1] * fx[1] + fx[2] * fx[2]);
    double s_minus = -pr;        // (a - foot).t
    double s_plus = len - pr;    // (b - foot).t
    double u0 = asinh(s_minus / dist), u1 = asinh(s_plus / dist);
    double half = 0.5 * (u1 - u0), mid = 0.5 * (u1 + u0);
    for (int q = 0; q < 32; ++q) {
      double u = mid + half * c_gl_x[q];
      double ch = cosh(u);
      double rho = dist * ch;
      double re, im;
      if (k == 0.0) {
        re = rho;
        im = 0.0;
      } else {
        double sh = sin(0.5 * k * rho);
        re = sin(k * rho) / k;
        im = 2.0 * sh * sh / k;
      }
      double wq = half * c_gl_w[q] / ch;
      acc.re += wq * re;
      acc.im += wq * im;
    }
  }
  return (1.0 / (4.0 * BEM_PI)) * acc;
}


// count / fill correction pairs.  One thread per sorted target.
__global__ void k_corr_pairs(int64_t nt, const double* __restrict__ cent, const double* __restrict__ hmax,
                             const int* __restrict__ elbox, const int* __restrict__ coll27,
                             const int* __restrict__ bstart, const int* __restrict__ bend, int pass, int* count,
                             const int* __restrict__ ptr, int* col) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nt) return;
  int b = elbox[i];
  double x0 = cent[3 * i], x1 = cent[3 * i + 1], x2 = cent[3 * i + 2];
  int n = 0, base = pass ? ptr[i] : 0;
  for (int t = 0; t < 27; ++t) {
    int c = coll27[27 * b + t];
    if (c < 0) continue;
    for (int j = bstart[c]; j < bend[c]; ++j) {
      double d0 = cent[3 * j] - x0, d1 = cent[3 * j + 1] - x1, d2 = cent[3 * j + 2] - x2;
      double dist2 = d0 * d0 + d1 * d1 + d2 * d2;
      double lim = 4.0 * hmax[j];
      if (j == i || dist2 < lim * lim) {
        if (pass) col[base + n] = j;
        ++n;
      }
    }
  }
  if (!pass) count[i] = n;
}

// correction values, one warp per target row; values divided by wgt[j].  The
// rules are summed in FP64 (the near-singular quadrature and the self term),
// and stored in the operator's precision (float4 in the mixed modes).  With
// rules32 (an option of the mixed modes) the rules of non-self pairs are
// summed in FP32 relative to the target instead, for a faster setup.
template <typename V4>
__global__ void k_corr_values(int64_t nt, double k, const double* __restrict__ cent, const double* __restrict__ qpt,
                              const double* __restrict__ nrm, const double* __restrict__ area,
                              const double* __restrict__ hmax, const double* __restrict__ wgt,
                              const int* __restrict__ ptr, const int* __restrict__ col, int rules32, V4* val) {
  int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
  int lane = threadIdx.x & 31;
  if (i >= nt) return;
  double x[3] = {cent[3 * i], cent[3 * i + 1], cent[3 * i + 2]};
  for (int e = ptr[i] + lane; e < ptr[i + 1]; e += 32) {
    int j = col[e];
    Tri64 t;
    load_tri64(qpt, nrm, cent, area, hmax, j, t);
    if (sizeof(V4) == sizeof(float4) && rules32 && (int64_t)j != i) {
      // mixed modes (values stored in FP32): both rules in FP32, target-relative
      double dd[3] = {t.c[0] - x[0], t.c[1] - x[1], t.c[2] - x[2]};
      double dist = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
      int L = dist < 2.0 * t.h ? 2 : (dist < 4.0 * t.h ? 1 : 0);
      V4 o;
      if (L == 0) {
        o.x = o.y = o.z = o.w = 0;
      } else {
        Tri32 tf;
        for (int a = 0; a < 3; ++a)
          for (int c = 0; c < 3; ++c) tf.v[a][c] = (float)(t.v[a][c] - x[c]);
        for (int c = 0; c < 3; ++c) tf.n[c] = (float)t.n[c];
        tf.area = (float)t.area;
        zf s0f = cmk(0.f, 0.f), d0f = s0f, s1f = s0f, d1f = s0f;
        rule_refined32(tf, 0, (float)k, s0f, d0f);
        rule_refined32(tf, L, (float)k, s1f, d1f);
        const float iwf = (float)(1.0 / wgt[j]);
        o.x = (s1f.re - s0f.re) * iwf;
        o.y = (s1f.im - s0f.im) * iwf;
        o.z = (d1f.re - d0f.re) * iwf;
        o.w = (d1f.im - d0f.im) * iwf;
      }
      val[e] = o;
      continue;
    }
    zd s0 = cmk(0.0, 0.0), d0 = cmk(0.0, 0.0), s1 = cmk(0.0, 0.0), d1 = cmk(0.0, 0.0);
    if ((int64_t)j == i) {
      // the near field leaves the pair of an element with itself out, so the
      // correction carries the whole exact self term
      s1 = self_single_layer(t, k);
      d1 = cmk(0.0, 0.0);
    } else {
      rule_refined(x, t, 0, k, s0, d0);  // what the regular rule contributes
      double dd[3] = {t.c[0] - x[0], t.c[1] - x[1], t.c[2] - x[2]};
      double dist = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
      int L = dist < 2.0 * t.h ? 2 : (dist < 4.0 * t.h ? 1 : 0);
      if (L == 0) {
        s1 = s0;
        d1 = d0;
      } else {
        rule_refined(x, t, L, k, s1, d1);
      }
    }
    double iw = 1.0 / wgt[j];
    V4 o;
    o.x = (s1.re - s0.re) * iw;
    o.y = (s1.im - s0.im) * iw;
    o.z = (d1.re - d0.re) * iw;
    o.w = (d1.im - d0.im) * iw;
    val[e] = o;
  }
}

// P2P arrays: sources relative to their leaf centre, normal components in .w
template <typename V4, typename R>
__global__ void k_p2p_arrays(int64_t nt, const double* __restrict__ cent, const double* __restrict__ qpt,
                             const double* __restrict__ nrm, const double* __restrict__ hmax,
                             const int* __restrict__ elbox, const double* __restrict__ bcentre, int relative, V4* tgt,
                             V4* src) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nt) return;
  double o[3] = {0, 0, 0};
  if (relative) {
    int b = elbox[s];
    for (int d = 0; d < 3; ++d) o[d] = bcentre[3 * b + d];
  }
  V4 t;
  t.x = (R)(cent[3 * s] - o[0]);
  t.y = (R)(cent[3 * s + 1] - o[1]);
  t.z = (R)(cent[3 * s + 2] - o[2]);
  t.w = (R)(16.0 * hmax[s] * hmax[s]);  // (4 h)^2: within it a field point needs the refined rule
  tgt[s] = t;
  for (int q = 0; q < 3; ++q) {
    V4 v;
    v.x = (R)(qpt[9 * s + 3 * q] - o[0]);
    v.y = (R)(qpt[9 * s + 3 * q + 1] - o[1]);
    v.z = (R)(qpt[9 * s + 3 * q + 2] - o[2]);
    v.w = (R)nrm[3 * s + q];
    src[3 * s + q] = v;
  }
}

// ------------------------------------------------------------- host side --
static void gauss_legendre_host(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(BEM_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 200; ++it) {
      double p0 = 1.0, p1 = z;
      for (int m = 2; m <= n; ++m) {
        double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
        p0 = p1;
        p1 = p2;
      }
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) {
        p0 = 1.0;
        p1 = z;
        for (int m = 2; m <= n; ++m) {
          double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        break;
      }
    }
  }
}

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

int bem_build_geometry(bem_handle* h, const double* dV, const int32_t* dT, cudaStream_t s) {
  int64_t nt = h->nt;
  double *cent_o, *qpt_o, *nrm_o, *area_o, *hmax_o;
  BEM_CUDA(cudaMallocAsync((void**)&cent_o, nt * 3 * sizeof(double), s));
  BEM_CUDA(cudaMallocAsync((void**)&qpt_o, nt * 9 * sizeof(double), s));
  BEM_CUDA(cudaMallocAsync((void**)&nrm_o, nt * 3 * sizeof(double), s));
  BEM_CUDA(cudaMallocAsync((void**)&area_o, nt * sizeof(double), s));
  BEM_CUDA(cudaMallocAsync((void**)&hmax_o, nt * sizeof(double), s));
  k_geometry<<<nblk(nt, 256), 256, 0, s>>>(dV, dT, nt, h->nv, cent_o, qpt_o, nrm_o, area_o, hmax_o, h->d_err);
  BEM_CUDA(cudaGetLastError());

  // bounding box of the vertices -> root cube
  int nb = (int)std::min<int64_t>(1024, (h->nv + 255) / 256);
  double* bb;
  BEM_CUDA(cudaMallocAsync((void**)&bb, 6 * nb * sizeof(double), s));
  k_bbox<<<nb, 256, 0, s>>>(dV, h->nv, bb);
  std::vector<double> hb(6 * nb);
  BEM_CUDA(cudaMemcpyAsync(hb.data(), bb, 6 * nb * sizeof(double), cudaMemcpyDeviceToHost, s));
  BEM_CUDA(cudaStreamSynchronize(s));
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int b = 0; b < nb; ++b)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], hb[6 * b + d]);
      hi[d] = std::max(hi[d], hb[6 * b + 3 + d]);
    }
  double ext = 0.0;
  for (int d = 0; d < 3; ++d) {
    if (!std::isfinite(lo[d]) || !std::isfinite(hi[d])) return bem_fail(BEM_ERR_DEGENERATE_MESH, "non-finite vertex");
    ext = std::max(ext, hi[d] - lo[d]);
    h->root_c[d] = 0.5 * (lo[d] + hi[d]);
  }
  if (!(ext > 0.0)) return bem_fail(BEM_ERR_DEGENERATE_MESH, "mesh has zero extent");
  h->root_w = ext * (1.0 + 1e-6) + 1e-300;

  // Morton keys at the finest level and the sort
  double lo_r[3];
  for (int d = 0; d < 3; ++d) lo_r[d] = h->root_c[d] - 0.5 * h->root_w;
  double wfine = h->root_w / (1 << BEM_MAXLEV);
  uint32_t *keys_in, *keys;
  int *idx_in;
  BEM_CUDA(cudaMallocAsync((void**)&keys_in, nt * sizeof(uint32_t), s));
  BEM_CUDA(cudaMallocAsync((void**)&keys, nt * sizeof(uint32_t), s));
  BEM_CUDA(cudaMallocAsync((void**)&idx_in, nt * sizeof(int), s));
  BEM_TRY(bem_alloc(h, &h->perm, nt));
  k_morton<<<nblk(nt, 256), 256, 0, s>>>(cent_o, nt, lo_r[0], lo_r[1], lo_r[2], wfine, keys_in, idx_in);
  size_t tmp_bytes = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, keys_in, keys, idx_in, h->perm, (int)nt, 0, 30, s);
  void* tmp;
  BEM_CUDA(cudaMallocAsync(&tmp, tmp_bytes, s));
  BEM_CUDA(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, keys_in, keys, idx_in, h->perm, (int)nt, 0, 30, s));

  // sorted geometry
  BEM_TRY(bem_alloc(h, &h->cent, nt * 3));
  BEM_TRY(bem_alloc(h, &h->qpt, nt * 9));
  BEM_TRY(bem_alloc(h, &h->nrm, nt * 3));
  BEM_TRY(bem_alloc(h, &h->area, nt));
  BEM_TRY(bem_alloc(h, &h->hmax, nt));
  BEM_TRY(bem_alloc(h, &h->wgt, nt));
  BEM_TRY(bem_alloc(h, &h->tri, nt * 3));
  k_permute_geometry<<<nblk(nt, 256), 256, 0, s>>>(h->perm, nt, cent_o, qpt_o, nrm_o, area_o, hmax_o, dT, h->cent,
                                                   h->qpt, h->nrm, h->area, h->hmax, h->wgt, h->tri);
  BEM_CUDA(cudaGetLastError());
  // longest edge over the mesh
  {
    double* dmax;
    BEM_CUDA(cudaMallocAsync((void**)&dmax, sizeof(double), s));
    size_t tb = 0;
    cub::DeviceReduce::Max(nullptr, tb, h->hmax, dmax, (int)nt, s);
    void* t2;
    BEM_CUDA(cudaMallocAsync(&t2, tb, s));
    BEM_CUDA(cub::DeviceReduce::Max(t2, tb, h->hmax, dmax, (int)nt, s));
    BEM_CUDA(cudaMemcpyAsync(&h->hmax_all, dmax, sizeof(double), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaFreeAsync(t2, s));
    BEM_CUDA(cudaFreeAsync(dmax, s));
  }
  // keep the sorted keys for the tree build (temporarily in the handle's alloc list)
  uint32_t* keys_keep;
  BEM_TRY(bem_alloc(h, &keys_keep, nt));
  BEM_CUDA(cudaMemcpyAsync(keys_keep, keys, nt * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  h->lev.assign(BEM_MAXLEV + 1, LevelInfo());
  h->lev[0].key = keys_keep;  // parked here until bem_build_tree replaces it

  BEM_CUDA(cudaFreeAsync(tmp, s));
  BEM_CUDA(cudaFreeAsync(keys_in, s));
  BEM_CUDA(cudaFreeAsync(keys, s));
  BEM_CUDA(cudaFreeAsync(idx_in, s));
  BEM_CUDA(cudaFreeAsync(bb, s));
  BEM_CUDA(cudaFreeAsync(cent_o, s));
  BEM_CUDA(cudaFreeAsync(qpt_o, s));
  BEM_CUDA(cudaFreeAsync(nrm_o, s));
  BEM_CUDA(cudaFreeAsync(area_o, s));
  BEM_CUDA(cudaFreeAsync(hmax_o, s));
  BEM_CUDA(cudaStreamSynchronize(s));
  return bem_check_device_error(h, s);
}

// ---------------------------------------------------------- adaptive tree --
namespace {
struct HostLevel {
  int nbox = 0;
  std::vector<uint32_t> key;
  std::vector<int> start, end, parent, child0, nchild, coord, coll;
  std::vector<double> centre, hm;
  std::vector<unsigned char> intree, internal;
};

// boxes (l1, c1) and (l2, c2) from different subtrees touch (share a face,
// edge or corner): their closed extents, on the finer level's grid, intersect
bool boxes_touch(int l1, const int* c1, int l2, const int* c2) {
  const int m = std::max(l1, l2);
  const int64_t s1 = int64_t(1) << (m - l1), s2 = int64_t(1) << (m - l2);
  for (int d = 0; d < 3; ++d) {
    const int64_t lo1 = c1[d] * s1, hi1 = lo1 + s1, lo2 = c2[d] * s2, hi2 = lo2 + s2;
    if (lo1 > hi2 || lo2 > hi1) return false;
  }
  return true;
}
}  // namespace

LevTab bem_levtab(const bem_handle* h) {
  LevTab t;
  for (int l = 0; l <= BEM_MAXLEV; ++l) {
    const bool has = l < (int)h->lev.size() && l >= 2 && l <= h->L;
    t.P[l] = has ? h->lev[l].P : 0;
    t.base[l] = has ? h->lev[l].exp_base : 0;
  }
  return t;
}

int bem_build_tree(bem_handle* h, int leaf_level, int leaf_target, cudaStream_t s) {
  int64_t nt = h->nt;
  uint32_t* keys = h->lev[0].key;
  double lo_r[3];
  for (int d = 0; d < 3; ++d) lo_r[d] = h->root_c[d] - 0.5 * h->root_w;

  // occupied boxes per level
  unsigned long long* dcnt;
  BEM_CUDA(cudaMallocAsync((void**)&dcnt, (BEM_MAXLEV + 1) * sizeof(unsigned long long), s));
  BEM_CUDA(cudaMemsetAsync(dcnt, 0, (BEM_MAXLEV + 1) * sizeof(unsigned long long), s));
  k_count_levels<<<nblk(nt, 256), 256, 0, s>>>(keys, nt, dcnt);
  unsigned long long cnt[BEM_MAXLEV + 1];
  BEM_CUDA(cudaMemcpyAsync(cnt, dcnt, sizeof(cnt), cudaMemcpyDeviceToHost, s));
  BEM_CUDA(cudaStreamSynchronize(s));
  BEM_CUDA(cudaFreeAsync(dcnt, s));

  // Uniform tree (leaf_level > 0): every box of that level is a leaf.
  // Adaptive trees: levels 0 and 1 are always split, and no box is split into
  // children narrower than 3 of its longest edges (quadrature points stay
  // close to their box, so expansions about the box centre converge one box
  // away).  leaf_level = -1: the depth is chosen per level-2 region, the
  // deepest level whose mean occupancy inside the region reaches leaf_target,
  // so leaves differ in level only between regions of different density and
  // the W/X-lists stay short.  leaf_level = -2: each box of level >= 2 is
  // split while it holds more than `split` elements.  If even level 2 is too
  // narrow for the longest edge, or the mesh fits one leaf, the tree is the
  // root alone and everything is near field.
  // leaf_level 0: the uniform level the whole mesh's mean occupancy picks
  // (the deepest level whose mean occupancy reaches leaf_target and whose
  // boxes are at least 3 longest edges wide; a level-1 leaf has no far field,
  // so that case keeps the single box)
  if (leaf_level == 0) {
    int Lauto = 0;
    for (int l = 0; l <= BEM_MAXLEV; ++l) {
      double wl = h->root_w / (1 << l);
      if ((double)nt / (double)cnt[l] >= (double)leaf_target && wl >= 3.0 * h->hmax_all) Lauto = l;
    }
    if (Lauto == 1) Lauto = 0;
    leaf_level = std::max(Lauto, 0);
  }
  const bool adaptive = leaf_level < 0;
  const bool regional = leaf_level == -1;
  const int split = 2 * std::max(leaf_target, 1);
  h->adaptive = adaptive ? (regional ? 1 : 2) : 0;
  // regional depth: distinct boxes per (level-2 region, level) from the sorted keys
  std::vector<int> region_depth;
  if (regional && !(h->root_w / 4.0 < 3.0 * h->hmax_all || nt <= split)) {
    std::vector<uint32_t> hk(nt);
    std::vector<double> hh(nt);
    BEM_CUDA(cudaMemcpyAsync(hk.data(), keys, nt * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaMemcpyAsync(hh.data(), h->hmax, nt * sizeof(double), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    const int R = 2, nreg = 1 << (3 * R);
    const int shR = 3 * (BEM_MAXLEV - R);
    std::vector<int64_t> nel(nreg, 0);
    std::vector<double> hreg(nreg, 0.0);
    std::vector<std::vector<int64_t>> nbox(BEM_MAXLEV + 1, std::vector<int64_t>(nreg, 0));
    for (int64_t i = 0; i < nt; ++i) {
      const int reg = (int)(hk[i] >> shR);
      ++nel[reg];
      hreg[reg] = std::max(hreg[reg], hh[i]);
      for (int l = R; l <= BEM_MAXLEV; ++l) {
        const int sh = 3 * (BEM_MAXLEV - l);
        if (i == 0 || (hk[i] >> sh) != (hk[i - 1] >> sh)) ++nbox[l][reg];
      }
    }
    region_depth.assign(nreg, R);
    for (int reg = 0; reg < nreg; ++reg) {
      if (nel[reg] == 0) continue;
      for (int l = R; l <= BEM_MAXLEV; ++l)
        if ((double)nel[reg] >= (double)leaf_target * (double)nbox[l][reg] &&
            h->root_w / (1 << l) >= 3.0 * hreg[reg])
          region_depth[reg] = l;
    }
  }
  int Lfix = std::min(std::max(leaf_level, 0), BEM_MAXLEV);  // 0 here: the single root box
  bool single = false;
  if (adaptive && (h->root_w / 4.0 < 3.0 * h->hmax_all || nt <= split)) single = true;

  int* flags;
  int* scan;
  BEM_CUDA(cudaMallocAsync((void**)&flags, nt * sizeof(int), s));
  BEM_CUDA(cudaMallocAsync((void**)&scan, nt * sizeof(int), s));
  size_t tb = 0;
  cub::DeviceScan::InclusiveSum(nullptr, tb, flags, scan, (int)nt, s);
  void* tmp;
  BEM_CUDA(cudaMallocAsync(&tmp, tb, s));
  std::vector<int*> elbox(BEM_MAXLEV + 1, nullptr);
  std::vector<HostLevel> hl(BEM_MAXLEV + 1);
  double* dhm = nullptr;
  BEM_CUDA(cudaMallocAsync((void**)&dhm, std::max<unsigned long long>(cnt[BEM_MAXLEV], 1) * sizeof(double), s));
  int L = 0;
  for (int l = 0; l <= BEM_MAXLEV; ++l) {
    LevelInfo& lv = h->lev[l];
    lv.nbox = (int)cnt[l];
    lv.w = h->root_w / (1 << l);
    int sh = 3 * (BEM_MAXLEV - l);
    BEM_TRY(bem_alloc(h, &elbox[l], nt));
    uint32_t* bkey;
    BEM_TRY(bem_alloc(h, &bkey, lv.nbox));
    BEM_TRY(bem_alloc(h, &lv.start, lv.nbox));
    BEM_TRY(bem_alloc(h, &lv.end, lv.nbox));
    BEM_TRY(bem_alloc(h, &lv.coord, 3 * lv.nbox));
    BEM_TRY(bem_alloc(h, &lv.centre, 3 * lv.nbox));
    BEM_TRY(bem_alloc(h, &lv.parent, lv.nbox));
    BEM_TRY(bem_alloc(h, &lv.child0, lv.nbox));
    BEM_TRY(bem_alloc(h, &lv.nchild, lv.nbox));
    BEM_TRY(bem_alloc(h, &lv.intree, lv.nbox));
    BEM_TRY(bem_alloc(h, &lv.internal, lv.nbox));
    k_level_flags<<<nblk(nt, 256), 256, 0, s>>>(keys, nt, sh, flags);
    BEM_CUDA(cub::DeviceScan::InclusiveSum(tmp, tb, flags, scan, (int)nt, s));
    k_level_boxes<<<nblk(nt, 256), 256, 0, s>>>(keys, scan, nt, sh, l, lo_r[0], lo_r[1], lo_r[2], lv.w, elbox[l], bkey,
                                                lv.start, lv.end, lv.coord, lv.centre);
    BEM_CUDA(cudaGetLastError());
    lv.key = bkey;  // (level 0 held the fine keys until now; `keys` still points at them)
    k_box_hmax<<<lv.nbox, 128, 0, s>>>(lv.nbox, lv.start, lv.end, h->hmax, dhm);
    BEM_CUDA(cudaGetLastError());
    HostLevel& H = hl[l];
    H.nbox = lv.nbox;
    H.key.resize(lv.nbox);
    H.start.resize(lv.nbox);
    H.end.resize(lv.nbox);
    H.coord.resize(3 * (size_t)lv.nbox);
    H.centre.resize(3 * (size_t)lv.nbox);
    H.hm.resize(lv.nbox);
    BEM_CUDA(cudaMemcpyAsync(H.key.data(), bkey, lv.nbox * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaMemcpyAsync(H.start.data(), lv.start, lv.nbox * sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaMemcpyAsync(H.end.data(), lv.end, lv.nbox * sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaMemcpyAsync(H.coord.data(), lv.coord, 3 * lv.nbox * sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaMemcpyAsync(H.centre.data(), lv.centre, 3 * lv.nbox * sizeof(double), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaMemcpyAsync(H.hm.data(), dhm, lv.nbox * sizeof(double), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    // parents on the host: the box of level l - 1 whose key is this key's prefix
    H.parent.assign(lv.nbox, -1);
    if (l > 0) {
      const std::vector<uint32_t>& pk = hl[l - 1].key;
      for (int b = 0; b < lv.nbox; ++b)
        H.parent[b] = (int)(std::lower_bound(pk.begin(), pk.end(), H.key[b] >> 3) - pk.begin());
    }
    // tree membership and leaf decision
    H.intree.assign(lv.nbox, 0);
    H.internal.assign(lv.nbox, 0);
    bool any_internal = false;
    const double wchild = h->root_w / (1 << (l + 1));
    for (int b = 0; b < lv.nbox; ++b) {
      const bool in = (l == 0) || hl[l - 1].internal[H.parent[b]] != 0;
      H.intree[b] = in ? 1 : 0;
      if (!in) continue;
      bool leaf;
      if (!adaptive)
        leaf = l >= Lfix;  // (Lfix = 0: the root alone)
      else if (single)
        leaf = true;
      else if (l < 2)
        leaf = false;
      else if (regional)
        leaf = l >= region_depth[H.key[b] >> (3 * (l - 2))];
      else
        leaf = l == BEM_MAXLEV || (H.end[b] - H.start[b]) <= split || wchild < 3.0 * H.hm[b];
      H.internal[b] = leaf ? 0 : 1;
      any_internal = any_internal || !leaf;
    }
    BEM_CUDA(cudaMemcpyAsync(lv.intree, H.intree.data(), lv.nbox, cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyAsync(lv.internal, H.internal.data(), lv.nbox, cudaMemcpyHostToDevice, s));
    L = l;
    if (!any_internal) break;
  }
  BEM_CUDA(cudaStreamSynchronize(s));
  BEM_CUDA(cudaFreeAsync(dhm, s));
  for (int l = L + 1; l <= BEM_MAXLEV; ++l) h->lev[l].nbox = 0;
  h->L = L;

  // the off-surface walk's far test per box: (4 h_max(box) / w_L)^2
  {
    const double wL = h->root_w / (1 << L);
    for (int l = 0; l <= L; ++l) {
      LevelInfo& lv = h->lev[l];
      std::vector<float> g2(lv.nbox);
      for (int b = 0; b < lv.nbox; ++b) {
        const double q = 4.0 * hl[l].hm[b] / wL;
        g2[b] = (float)(q * q);
      }
      BEM_TRY(bem_alloc(h, &lv.gap2, lv.nbox));
      BEM_CUDA(cudaMemcpyAsync(lv.gap2, g2.data(), lv.nbox * sizeof(float), cudaMemcpyHostToDevice, s));
      BEM_CUDA(cudaStreamSynchronize(s));
    }
  }

  // near-singular search level: widest boxes still >= 4 h_max
  int Lc = 0;
  for (int l = 0; l <= L; ++l)
    if (h->root_w / (1 << l) >= 4.0 * h->hmax_all) Lc = l;
  h->Lc = Lc;

  for (int l = 0; l <= L; ++l) {
    LevelInfo& lv = h->lev[l];
    k_level_links<<<nblk(lv.nbox, 128), 128, 0, s>>>(lv.nbox, lv.start, lv.end, l > 0 ? elbox[l - 1] : nullptr,
                                                     l < L ? elbox[l + 1] : nullptr, lv.parent, lv.child0, lv.nchild);
    BEM_CUDA(cudaGetLastError());
  }

  // colleagues on every level (V-lists, the near-field lists, correction search)
  std::vector<int*> coll(L + 1);
  for (int l = 0; l <= L; ++l) {
    BEM_TRY(bem_alloc(h, &coll[l], 27 * (size_t)h->lev[l].nbox));
    k_colleagues<<<nblk(h->lev[l].nbox, 128), 128, 0, s>>>(h->lev[l].nbox, h->lev[l].key, h->lev[l].coord, 1 << l,
                                                           coll[l]);
    BEM_CUDA(cudaGetLastError());
  }
  for (int l = 0; l <= L; ++l) {
    HostLevel& H = hl[l];
    H.coll.resize(27 * (size_t)H.nbox);
    H.child0.resize(H.nbox);
    H.nchild.resize(H.nbox);
    BEM_CUDA(cudaMemcpyAsync(H.coll.data(), coll[l], H.coll.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaMemcpyAsync(H.child0.data(), h->lev[l].child0, H.nbox * sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaMemcpyAsync(H.nchild.data(), h->lev[l].nchild, H.nbox * sizeof(int), cudaMemcpyDeviceToHost, s));
  }
  BEM_CUDA(cudaStreamSynchronize(s));

  // ---- leaves, numbered level by level ----
  std::vector<int> gl_level, gl_box;
  for (int l = 0; l <= L; ++l) {
    LevelInfo& lv = h->lev[l];
    HostLevel& H = hl[l];
    std::vector<int> lb;
    for (int b = 0; b < H.nbox; ++b)
      if (H.intree[b] && !H.internal[b]) lb.push_back(b);
    lv.nleaf = (int)lb.size();
    lv.leaf_g0 = (int)gl_level.size();
    for (int b : lb) {
      gl_level.push_back(l);
      gl_box.push_back(b);
    }
    BEM_TRY(bem_alloc(h, &lv.leafbox, std::max<size_t>(lb.size(), 1)));
    if (!lb.empty())
      BEM_CUDA(cudaMemcpyAsync(lv.leafbox, lb.data(), lb.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaStreamSynchronize(s));
  }
  const int ng = (int)gl_level.size();
  h->nleaf_all = ng;
  std::vector<int> hgs(ng), hge(ng);
  std::vector<double> hgc(3 * (size_t)ng);
  std::vector<std::vector<int>> gid(L + 1);
  for (int l = 0; l <= L; ++l) gid[l].assign(hl[l].nbox, -1);
  for (int g = 0; g < ng; ++g) {
    const int l = gl_level[g], b = gl_box[g];
    hgs[g] = hl[l].start[b];
    hge[g] = hl[l].end[b];
    for (int d = 0; d < 3; ++d) hgc[3 * (size_t)g + d] = hl[l].centre[3 * (size_t)b + d];
    gid[l][b] = g;
  }
  BEM_TRY(bem_alloc(h, &h->gl_start, std::max(ng, 1)));
  BEM_TRY(bem_alloc(h, &h->gl_end, std::max(ng, 1)));
  double* d_glc;
  BEM_TRY(bem_alloc(h, &d_glc, 3 * (size_t)std::max(ng, 1)));
  BEM_CUDA(cudaMemcpyAsync(h->gl_start, hgs.data(), ng * sizeof(int), cudaMemcpyHostToDevice, s));
  BEM_CUDA(cudaMemcpyAsync(h->gl_end, hge.data(), ng * sizeof(int), cudaMemcpyHostToDevice, s));
  BEM_CUDA(cudaMemcpyAsync(d_glc, hgc.data(), hgc.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  BEM_TRY(bem_alloc(h, &h->leaf_of, nt));
  BEM_TRY(bem_alloc(h, &h->leaf_lev, nt));
  BEM_TRY(bem_alloc(h, &h->gleaf_of, nt));
  for (int l = 0; l <= L; ++l) {
    LevelInfo& lv = h->lev[l];
    if (lv.nleaf == 0) continue;
    k_leaf_mark<<<lv.nleaf, 128, 0, s>>>(lv.nleaf, lv.leafbox, lv.start, lv.end, l, lv.leaf_g0, h->leaf_of,
                                         h->leaf_lev, h->gleaf_of);
    BEM_CUDA(cudaGetLastError());
  }

  // ---- U-, W- and X-lists on the host ----
  // For leaf g of level l: U(g) holds every leaf that touches g (g included);
  // W(g) holds the boxes D below g's colleagues that do not touch g although
  // their parents do (D's multipole converges on g); X(D) gets g in return
  // (g's elements expanded about D's centre).  Together with the V-lists of g
  // and its ancestors this counts every (target, source) pair exactly once.
  std::vector<int> uptr(ng + 1, 0), usrc, wptr(ng + 1, 0), wsrc;
  std::vector<double> ushift, wshift;
  std::vector<std::vector<int>> xdst(L + 1), xsrc(L + 1);
  std::vector<std::vector<double>> xshift(L + 1);
  auto push_u = [&](int g, int lsrc, int bsrc) {
    const int gs = gid[lsrc][bsrc];
    usrc.push_back(gs);
    for (int d = 0; d < 3; ++d) ushift.push_back(hgc[3 * (size_t)gs + d] - hgc[3 * (size_t)g + d]);
  };
  for (int g = 0; g < ng; ++g) {
    const int l = gl_level[g], b = gl_box[g];
    const int* cb = &hl[l].coord[3 * (size_t)b];
    if (l == 0) push_u(g, l, b);
    if (l > 0) {
      // same-level colleagues in slot order (g itself in the middle slot),
      // and the tree below the internal ones
      std::vector<std::pair<int, int>> stack;
      for (int t = 0; t < 27; ++t) {
        if (t == 13) {
          push_u(g, l, b);
          continue;
        }
        const int c = hl[l].coll[27 * (size_t)b + t];
        if (c < 0 || !hl[l].intree[c]) continue;
        if (!hl[l].internal[c])
          push_u(g, l, c);
        else
          stack.push_back({l, c});
      }
      while (!stack.empty()) {
        const auto [m, dbox] = stack.back();
        stack.pop_back();
        for (int ch = hl[m].child0[dbox]; ch < hl[m].child0[dbox] + hl[m].nchild[dbox]; ++ch) {
          if (boxes_touch(m + 1, &hl[m + 1].coord[3 * (size_t)ch], l, cb)) {
            if (hl[m + 1].internal[ch])
              stack.push_back({m + 1, ch});
            else
              push_u(g, m + 1, ch);
          } else {
            wsrc.push_back(((m + 1) << 24) | ch);
            for (int d = 0; d < 3; ++d)
              wshift.push_back(hgc[3 * (size_t)g + d] - hl[m + 1].centre[3 * (size_t)ch + d]);
            xdst[m + 1].push_back(ch);
            xsrc[m + 1].push_back(g);
            for (int d = 0; d < 3; ++d)
              xshift[m + 1].push_back(hgc[3 * (size_t)g + d] - hl[m + 1].centre[3 * (size_t)ch + d]);
          }
        }
      }
      // coarser leaves that touch g: colleagues of g's ancestors
      int a = b;
      for (int la = l - 1; la >= 0; --la) {
        a = hl[la + 1].parent[a];
        for (int t = 0; t < 27; ++t) {
          if (t == 13) continue;
          const int c = hl[la].coll[27 * (size_t)a + t];
          if (c < 0 || !hl[la].intree[c] || hl[la].internal[c]) continue;
          if (boxes_touch(la, &hl[la].coord[3 * (size_t)c], l, cb)) push_u(g, la, c);
        }
      }
    }
    uptr[g + 1] = (int)usrc.size();
    wptr[g + 1] = (int)wsrc.size();
  }
  h->u_nnz = (int64_t)usrc.size();
  h->w_nnz = (int)wsrc.size();
  BEM_TRY(bem_alloc(h, &h->u_ptr, ng + 1));
  BEM_TRY(bem_alloc(h, &h->u_src, std::max<size_t>(usrc.size(), 1)));
  BEM_TRY(bem_alloc(h, &h->w_ptr, ng + 1));
  BEM_TRY(bem_alloc(h, &h->w_src, std::max<size_t>(wsrc.size(), 1)));
  BEM_CUDA(cudaMemcpyAsync(h->u_ptr, uptr.data(), (ng + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  BEM_CUDA(cudaMemcpyAsync(h->u_src, usrc.data(), usrc.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  BEM_CUDA(cudaMemcpyAsync(h->w_ptr, wptr.data(), (ng + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  if (!wsrc.empty())
    BEM_CUDA(cudaMemcpyAsync(h->w_src, wsrc.data(), wsrc.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  std::vector<int> wl;
  for (int g = 0; g < ng; ++g)
    if (wptr[g + 1] > wptr[g]) wl.push_back(g);
  h->n_w_leaves = (int)wl.size();
  BEM_TRY(bem_alloc(h, &h->w_leaves, std::max<size_t>(wl.size(), 1)));
  if (!wl.empty())
    BEM_CUDA(cudaMemcpyAsync(h->w_leaves, wl.data(), wl.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  // offsets in the operator's precision
  auto upload_shift = [&](const std::vector<double>& v, float4** f, double4** d) -> int {
    const size_t n = v.size() / 3;
    if (bem_is_fp64(h)) {
      std::vector<double4> o(std::max<size_t>(n, 1));
      for (size_t i = 0; i < n; ++i) o[i] = make_double4(v[3 * i], v[3 * i + 1], v[3 * i + 2], 0.0);
      BEM_TRY(bem_alloc(h, d, o.size()));
      BEM_CUDA(cudaMemcpyAsync(*d, o.data(), o.size() * sizeof(double4), cudaMemcpyHostToDevice, s));
    } else {
      std::vector<float4> o(std::max<size_t>(n, 1));
      for (size_t i = 0; i < n; ++i)
        o[i] = make_float4((float)v[3 * i], (float)v[3 * i + 1], (float)v[3 * i + 2], 0.f);
      BEM_TRY(bem_alloc(h, f, o.size()));
      BEM_CUDA(cudaMemcpyAsync(*f, o.data(), o.size() * sizeof(float4), cudaMemcpyHostToDevice, s));
    }
    BEM_CUDA(cudaStreamSynchronize(s));
    return BEM_OK;
  };
  BEM_TRY(upload_shift(ushift, &h->u_shift32, &h->u_shift64));
  BEM_TRY(upload_shift(wshift, &h->w_shift32, &h->w_shift64));
  for (int l = 0; l <= L; ++l) {
    h->x_n[l] = (int)xdst[l].size();
    if (xdst[l].empty()) continue;
    BEM_TRY(bem_alloc(h, &h->x_dst[l], xdst[l].size()));
    BEM_TRY(bem_alloc(h, &h->x_src[l], xsrc[l].size()));
    BEM_CUDA(cudaMemcpyAsync(h->x_dst[l], xdst[l].data(), xdst[l].size() * sizeof(int), cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyAsync(h->x_src[l], xsrc[l].data(), xsrc[l].size() * sizeof(int), cudaMemcpyHostToDevice, s));
    BEM_TRY(upload_shift(xshift[l], &h->x_shift32[l], &h->x_shift64[l]));
    for (size_t i = 0; i < xsrc[l].size(); ++i) h->x_pts[l] += 3 * (int64_t)(hge[xsrc[l][i]] - hgs[xsrc[l][i]]);
  }
  for (int g = 0; g < ng; ++g)
    for (int e = wptr[g]; e < wptr[g + 1]; ++e) h->w_tp[wsrc[e] >> 24] += hge[g] - hgs[g];

  // ---- P2P work units: each leaf's targets cut into blocks of p2p_unit
  // targets plus the binary decomposition of the remainder, sorted by cost ----
  {
    const int U = h->p2p_unit, ulog = U == 16 ? 4 : (U == 32 ? 5 : 6);
    std::vector<std::pair<int64_t, int4>> units;
    int64_t pairs = 0;
    for (int g = 0; g < ng; ++g) {
      int64_t ns = 0;
      for (int e = uptr[g]; e < uptr[g + 1]; ++e) ns += hge[usrc[e]] - hgs[usrc[e]];
      int t0 = hgs[g], nc = hge[g] - hgs[g];
      pairs += ns * nc;
      while (nc >= U) {
        units.push_back({U * ns, make_int4(g, t0, U, 0)});
        t0 += U;
        nc -= U;
      }
      for (int j = ulog - 1; j >= 0; --j)
        if (nc & (1 << j)) {
          units.push_back({(int64_t)(1 << j) * ns, make_int4(g, t0, 1 << j, 0)});
          t0 += 1 << j;
        }
    }
    h->p2p_pairs = pairs;
    std::stable_sort(units.begin(), units.end(),
                     [](const std::pair<int64_t, int4>& a, const std::pair<int64_t, int4>& b) { return a.first > b.first; });
    std::vector<int4> u4(units.size());
    for (size_t i = 0; i < units.size(); ++i) u4[i] = units[i].second;
    h->n_p2p_units = (int)u4.size();
    BEM_TRY(bem_alloc(h, &h->p2p_units, std::max<size_t>(u4.size(), 1)));
    BEM_CUDA(cudaMemcpyAsync(h->p2p_units, u4.data(), u4.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaStreamSynchronize(s));
  }

  // ---- correction pairs (FP64 values) ----
  {
    int* cntr;
    BEM_TRY(bem_alloc(h, &h->corr_ptr, nt + 1));
    BEM_CUDA(cudaMallocAsync((void**)&cntr, (nt + 1) * sizeof(int), s));
    BEM_CUDA(cudaMemsetAsync(cntr, 0, (nt + 1) * sizeof(int), s));
    LevelInfo& lc = h->lev[Lc];
    k_corr_pairs<<<nblk(nt, 128), 128, 0, s>>>(nt, h->cent, h->hmax, elbox[Lc], coll[Lc], lc.start, lc.end, 0, cntr,
                                               nullptr, nullptr);
    size_t tb2 = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, tb2, cntr, h->corr_ptr, (int)nt + 1, s);
    void* t2;
    BEM_CUDA(cudaMallocAsync(&t2, tb2, s));
    BEM_CUDA(cub::DeviceScan::ExclusiveSum(t2, tb2, cntr, h->corr_ptr, (int)nt + 1, s));
    int nnz = 0;
    BEM_CUDA(cudaMemcpyAsync(&nnz, h->corr_ptr + nt, sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    h->corr_nnz = nnz;
    BEM_TRY(bem_alloc(h, &h->corr_col, nnz));
    k_corr_pairs<<<nblk(nt, 128), 128, 0, s>>>(nt, h->cent, h->hmax, elbox[Lc], coll[Lc], lc.start, lc.end, 1, nullptr,
                                               h->corr_ptr, h->corr_col);
    BEM_CUDA(cudaGetLastError());
    double glx[32], glw[32];
    gauss_legendre_host(32, glx, glw);
    BEM_CUDA(cudaMemcpyToSymbolAsync(c_gl_x, glx, sizeof(glx), 0, cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyToSymbolAsync(c_gl_w, glw, sizeof(glw), 0, cudaMemcpyHostToDevice, s));
    if (bem_is_fp64(h)) {
      double4* v;
      BEM_TRY(bem_alloc(h, &v, nnz));
      h->corr_val = v;
      k_corr_values<double4><<<nblk(nt * 32, 128), 128, 0, s>>>(nt, h->k, h->cent, h->qpt, h->nrm, h->area, h->hmax,
                                                                 h->wgt, h->corr_ptr, h->corr_col, 0, v);
    } else {
      float4* v;
      BEM_TRY(bem_alloc(h, &v, nnz));
      h->corr_val = v;
      k_corr_values<float4><<<nblk(nt * 32, 128), 128, 0, s>>>(nt, h->k, h->cent, h->qpt, h->nrm, h->area, h->hmax,
                                                                h->wgt, h->corr_ptr, h->corr_col, h->corr_rules32, v);
    }
    BEM_CUDA(cudaGetLastError());
    BEM_CUDA(cudaFreeAsync(t2, s));
    BEM_CUDA(cudaFreeAsync(cntr, s));
  }

  // ---- P2P arrays ----
  // FMM: coordinates relative to the element's leaf centre (keeps FP32
  // differences accurate; the kernels add the exact offset between leaf
  // centres).  Direct sums: one common frame, the root centre.
  bool direct = (h->mode == BEM_MODE_DIRECT_FP64 || h->mode == BEM_MODE_DIRECT_FP32);
  {
    const int* frame_of = h->gleaf_of;
    const double* frame_c = d_glc;
    double* rc = nullptr;
    int* zero = nullptr;
    if (direct) {
      BEM_CUDA(cudaMallocAsync((void**)&rc, 3 * sizeof(double), s));
      BEM_CUDA(cudaMemcpyAsync(rc, h->root_c, 3 * sizeof(double), cudaMemcpyHostToDevice, s));
      BEM_CUDA(cudaMallocAsync((void**)&zero, nt * sizeof(int), s));
      BEM_CUDA(cudaMemsetAsync(zero, 0, nt * sizeof(int), s));
      frame_of = zero;
      frame_c = rc;
    }
    if (bem_is_fp64(h)) {
      BEM_TRY(bem_alloc(h, &h->tgt64, nt));
      BEM_TRY(bem_alloc(h, &h->src64, 3 * nt));
      k_p2p_arrays<double4, double><<<nblk(nt, 256), 256, 0, s>>>(nt, h->cent, h->qpt, h->nrm, h->hmax, frame_of,
                                                                  frame_c, 1, h->tgt64, h->src64);
    } else {
      BEM_TRY(bem_alloc(h, &h->tgt32, nt));
      BEM_TRY(bem_alloc(h, &h->src32, 3 * nt));
      k_p2p_arrays<float4, float><<<nblk(nt, 256), 256, 0, s>>>(nt, h->cent, h->qpt, h->nrm, h->hmax, frame_of,
                                                                frame_c, 1, h->tgt32, h->src32);
    }
    BEM_CUDA(cudaGetLastError());
    BEM_CUDA(cudaStreamSynchronize(s));
    if (rc) BEM_CUDA(cudaFreeAsync(rc, s));
    if (zero) BEM_CUDA(cudaFreeAsync(zero, s));
  }

  // ---- V-lists (levels >= 2), grouped by offset ----
  for (int l = 2; l <= L && bem_is_fmm(h); ++l) {
    LevelInfo& lv = h->lev[l];
    LevelInfo& pv = h->lev[l - 1];
    int *dcnt2, *dcur, *dstart;
    BEM_CUDA(cudaMallocAsync((void**)&dcnt2, 343 * sizeof(int), s));
    BEM_CUDA(cudaMallocAsync((void**)&dcur, 343 * sizeof(int), s));
    BEM_CUDA(cudaMallocAsync((void**)&dstart, 344 * sizeof(int), s));
    BEM_CUDA(cudaMemsetAsync(dcnt2, 0, 343 * sizeof(int), s));
    BEM_CUDA(cudaMemsetAsync(dcur, 0, 343 * sizeof(int), s));
    k_vlist<<<nblk(lv.nbox, 128), 128, 0, s>>>(lv.nbox, lv.coord, lv.parent, coll[l - 1], pv.child0, pv.nchild,
                                               lv.coord, lv.intree, pv.internal, 0, dcnt2, nullptr, nullptr, nullptr,
                                               nullptr);
    int hc[343];
    BEM_CUDA(cudaMemcpyAsync(hc, dcnt2, sizeof(hc), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    std::vector<int> gs(344, 0);
    for (int o = 0; o < 343; ++o) gs[o + 1] = gs[o] + hc[o];
    int np = gs[343];
    GroupedOp& op = h->m2l[l];
    op.npairs = np;
    op.ngroups = 0;
    op.pair_start.clear();
    std::vector<int> goff;  // offset id per group
    for (int o = 0; o < 343; ++o)
      if (hc[o] > 0) {
        goff.push_back(o);
        op.pair_start.push_back(gs[o]);
      }
    op.pair_start.push_back(np);
    op.ngroups = (int)goff.size();
    op.codes = goff;
    int *src_box, *dst_box;
    BEM_TRY(bem_alloc(h, &op.d_src_off, std::max(np, 1)));
    BEM_TRY(bem_alloc(h, &op.d_dst_off, std::max(np, 1)));
    src_box = op.d_src_off;
    dst_box = op.d_dst_off;
    BEM_CUDA(cudaMemcpyAsync(dstart, gs.data(), 344 * sizeof(int), cudaMemcpyHostToDevice, s));
    k_vlist<<<nblk(lv.nbox, 128), 128, 0, s>>>(lv.nbox, lv.coord, lv.parent, coll[l - 1], pv.child0, pv.nchild,
                                               lv.coord, lv.intree, pv.internal, 1, nullptr, dcur, dstart, src_box,
                                               dst_box);
    BEM_CUDA(cudaGetLastError());
    BEM_CUDA(cudaStreamSynchronize(s));
    BEM_CUDA(cudaFreeAsync(dcnt2, s));
    BEM_CUDA(cudaFreeAsync(dcur, s));
    BEM_CUDA(cudaFreeAsync(dstart, s));
  }

  BEM_CUDA(cudaFreeAsync(flags, s));
  BEM_CUDA(cudaFreeAsync(scan, s));
  BEM_CUDA(cudaFreeAsync(tmp, s));
  BEM_CUDA(cudaStreamSynchronize(s));
  return bem_check_device_error(h, s);
}
