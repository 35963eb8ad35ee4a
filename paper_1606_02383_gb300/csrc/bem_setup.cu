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
// Near-singular correction: for every target i and source j with j == i or
// |x_i - c_j| < 4 h_j, C_ij = (entry by the refined rule R_L or the exact self
// term) - (entry by the regular rule R_0), for S and D, in FP64.  The apply
// evaluates R_0 for every pair (near field directly, far field by the FMM) and
// adds C, which reproduces the rule-defined operator.
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

// V-list: children of the parent's colleagues not adjacent to b.  pass 0 counts per offset, pass 1 fills.
__global__ void k_vlist(int nbox, const int* __restrict__ coord, const int* __restrict__ parent,
                        const int* __restrict__ pcoll27, const int* __restrict__ pchild0,
                        const int* __restrict__ pnchild, const int* __restrict__ ccoord, int pass, int* counts,
                        int* cursor, const int* __restrict__ gstart, int* src_box, int* dst_box) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  int p = parent[b];
  int bx = coord[3 * b], by = coord[3 * b + 1], bz = coord[3 * b + 2];
  for (int t = 0; t < 27; ++t) {
    int q = pcoll27[27 * p + t];
    if (q < 0) continue;
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

// correction values, one warp per target row; values divided by wgt[j].  In the
// FP64 modes everything is FP64; in the mixed modes (FP32 values) the rules of
// non-self pairs are summed in FP32 relative to the target, the self term in FP64.
template <typename V4>
__global__ void k_corr_values(int64_t nt, double k, const double* __restrict__ cent, const double* __restrict__ qpt,
                              const double* __restrict__ nrm, const double* __restrict__ area,
                              const double* __restrict__ hmax, const double* __restrict__ wgt,
                              const int* __restrict__ ptr, const int* __restrict__ col, V4* val) {
  int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
  int lane = threadIdx.x & 31;
  if (i >= nt) return;
  double x[3] = {cent[3 * i], cent[3 * i + 1], cent[3 * i + 2]};
  for (int e = ptr[i] + lane; e < ptr[i + 1]; e += 32) {
    int j = col[e];
    Tri64 t;
    load_tri64(qpt, nrm, cent, area, hmax, j, t);
    if (sizeof(V4) == sizeof(float4) && (int64_t)j != i) {
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
    rule_refined(x, t, 0, k, s0, d0);  // what the regular rule contributes
    if ((int64_t)j == i) {
      s1 = self_single_layer(t, k);
      d1 = cmk(0.0, 0.0);
    } else {
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
                             const double* __restrict__ nrm, const int* __restrict__ elbox,
                             const double* __restrict__ bcentre, int relative, V4* tgt, V4* src) {
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
  t.w = (R)0;
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

int bem_build_tree(bem_handle* h, int leaf_level, int leaf_target, cudaStream_t s) {
  int64_t nt = h->nt;
  uint32_t* keys = h->lev[0].key;
  double lo_r[3];
  for (int d = 0; d < 3; ++d) lo_r[d] = h->root_c[d] - 0.5 * h->root_w;

  // occupied boxes per level -> leaf level
  unsigned long long* dcnt;
  BEM_CUDA(cudaMallocAsync((void**)&dcnt, (BEM_MAXLEV + 1) * sizeof(unsigned long long), s));
  BEM_CUDA(cudaMemsetAsync(dcnt, 0, (BEM_MAXLEV + 1) * sizeof(unsigned long long), s));
  k_count_levels<<<nblk(nt, 256), 256, 0, s>>>(keys, nt, dcnt);
  unsigned long long cnt[BEM_MAXLEV + 1];
  BEM_CUDA(cudaMemcpyAsync(cnt, dcnt, sizeof(cnt), cudaMemcpyDeviceToHost, s));
  BEM_CUDA(cudaStreamSynchronize(s));
  BEM_CUDA(cudaFreeAsync(dcnt, s));
  int L;
  if (leaf_level > 0) {
    L = std::min(leaf_level, BEM_MAXLEV);
  } else {
    // deepest level whose mean occupancy reaches the target and whose boxes are at
    // least 3 longest edges wide (quadrature points stay close to their box)
    L = 0;
    for (int l = 0; l <= BEM_MAXLEV; ++l) {
      double wl = h->root_w / (1 << l);
      if ((double)nt / (double)cnt[l] >= (double)leaf_target && wl >= 3.0 * h->hmax_all) L = l;
    }
    if (L == 1) L = 0;  // a level-1 leaf has no far field either; keep the single box
  }
  h->L = L;

  // near-singular search level: widest boxes still >= 4 h_max
  int Lc = 0;
  for (int l = 0; l <= L; ++l)
    if (h->root_w / (1 << l) >= 4.0 * h->hmax_all) Lc = l;
  h->Lc = Lc;

  // boxes of every level 0..L
  int* flags;
  int* scan;
  BEM_CUDA(cudaMallocAsync((void**)&flags, nt * sizeof(int), s));
  BEM_CUDA(cudaMallocAsync((void**)&scan, nt * sizeof(int), s));
  size_t tb = 0;
  cub::DeviceScan::InclusiveSum(nullptr, tb, flags, scan, (int)nt, s);
  void* tmp;
  BEM_CUDA(cudaMallocAsync(&tmp, tb, s));
  std::vector<int*> elbox(L + 1);
  for (int l = 0; l <= L; ++l) {
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
    k_level_flags<<<nblk(nt, 256), 256, 0, s>>>(keys, nt, sh, flags);
    BEM_CUDA(cub::DeviceScan::InclusiveSum(tmp, tb, flags, scan, (int)nt, s));
    k_level_boxes<<<nblk(nt, 256), 256, 0, s>>>(keys, scan, nt, sh, l, lo_r[0], lo_r[1], lo_r[2], lv.w, elbox[l], bkey,
                                                lv.start, lv.end, lv.coord, lv.centre);
    BEM_CUDA(cudaGetLastError());
    lv.key = bkey;  // (level 0 held the fine keys until now; `keys` still points at them)
  }
  for (int l = 0; l <= L; ++l) {
    LevelInfo& lv = h->lev[l];
    k_level_links<<<nblk(lv.nbox, 128), 128, 0, s>>>(lv.nbox, lv.start, lv.end, l > 0 ? elbox[l - 1] : nullptr,
                                                     l < L ? elbox[l + 1] : nullptr, lv.parent, lv.child0, lv.nchild);
    BEM_CUDA(cudaGetLastError());
  }

  // colleagues on every level (needed for V-lists, near field and correction search)
  std::vector<int*> coll(L + 1);
  for (int l = 0; l <= L; ++l) {
    BEM_TRY(bem_alloc(h, &coll[l], 27 * (size_t)h->lev[l].nbox));
    k_colleagues<<<nblk(h->lev[l].nbox, 128), 128, 0, s>>>(h->lev[l].nbox, h->lev[l].key, h->lev[l].coord, 1 << l,
                                                           coll[l]);
    BEM_CUDA(cudaGetLastError());
  }
  h->near27 = coll[L];
  {
    unsigned long long* dp;
    BEM_CUDA(cudaMallocAsync((void**)&dp, sizeof(unsigned long long), s));
    BEM_CUDA(cudaMemsetAsync(dp, 0, sizeof(unsigned long long), s));
    k_count_p2p<<<nblk(h->lev[L].nbox, 128), 128, 0, s>>>(h->lev[L].nbox, coll[L], h->lev[L].start, h->lev[L].end, dp);
    unsigned long long v = 0;
    BEM_CUDA(cudaMemcpyAsync(&v, dp, sizeof(v), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    BEM_CUDA(cudaFreeAsync(dp, s));
    h->p2p_pairs = (int64_t)v;
  }
  // P2P warp work units: each leaf's targets cut into 64-target blocks plus the
  // binary decomposition of the remainder, sorted by cost (targets x near sources)
  if (bem_is_fmm(h)) {
    int nl = h->lev[L].nbox;
    std::vector<int> hs(nl), he(nl), hn(27 * (size_t)nl);
    BEM_CUDA(cudaMemcpyAsync(hs.data(), h->lev[L].start, nl * sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaMemcpyAsync(he.data(), h->lev[L].end, nl * sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaMemcpyAsync(hn.data(), coll[L], hn.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    std::vector<std::pair<int64_t, int4>> units;
    for (int b = 0; b < nl; ++b) {
      int64_t ns = 0;
      for (int t = 0; t < 27; ++t) {
        int c = hn[27 * (size_t)b + t];
        if (c >= 0) ns += he[c] - hs[c];
      }
      int t0 = hs[b], nc = he[b] - hs[b];
      while (nc >= 64) {
        units.push_back({64 * ns, make_int4(b, t0, 64, 0)});
        t0 += 64;
        nc -= 64;
      }
      for (int j = 5; j >= 0; --j)
        if (nc & (1 << j)) {
          units.push_back({(int64_t)(1 << j) * ns, make_int4(b, t0, 1 << j, 0)});
          t0 += 1 << j;
        }
    }
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
                                                                 h->wgt, h->corr_ptr, h->corr_col, v);
    } else {
      float4* v;
      BEM_TRY(bem_alloc(h, &v, nnz));
      h->corr_val = v;
      k_corr_values<float4><<<nblk(nt * 32, 128), 128, 0, s>>>(nt, h->k, h->cent, h->qpt, h->nrm, h->area, h->hmax,
                                                                h->wgt, h->corr_ptr, h->corr_col, v);
    }
    BEM_CUDA(cudaGetLastError());
    BEM_CUDA(cudaFreeAsync(t2, s));
    BEM_CUDA(cudaFreeAsync(cntr, s));
  }

  // ---- P2P arrays ----
  // FMM: coordinates relative to the element's leaf centre (keeps FP32
  // differences accurate; the kernel adds the exact box offset).  Direct sums:
  // one common frame, the root centre.
  bool direct = (h->mode == BEM_MODE_DIRECT_FP64 || h->mode == BEM_MODE_DIRECT_FP32);
  {
    const int* frame_of = elbox[L];
    const double* frame_c = h->lev[L].centre;
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
      k_p2p_arrays<double4, double><<<nblk(nt, 256), 256, 0, s>>>(nt, h->cent, h->qpt, h->nrm, frame_of, frame_c, 1,
                                                                  h->tgt64, h->src64);
    } else {
      BEM_TRY(bem_alloc(h, &h->tgt32, nt));
      BEM_TRY(bem_alloc(h, &h->src32, 3 * nt));
      k_p2p_arrays<float4, float><<<nblk(nt, 256), 256, 0, s>>>(nt, h->cent, h->qpt, h->nrm, frame_of, frame_c, 1,
                                                                h->tgt32, h->src32);
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
                                               lv.coord, 0, dcnt2, nullptr, nullptr, nullptr, nullptr);
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
                                               lv.coord, 1, nullptr, dcur, dstart, src_box, dst_box);
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
