// bem_adjoint.cu -- conjugate-transpose apply: gx = (1/2 I - D)^H g, gy = S^H g.
//
// The adjoint problem of Section 2.2 is solved with the same matrix as the
// state problem; this is the operator reverse-mode differentiation of
// bem_apply needs.  With h = conj(g) the two products are the plain
// transposes u = S^T h, v = D^T h, and gy = conj(u), gx = 1/2 g - conj(v).
// Every part of the forward operator is transposed:
//   near field   u_j += sum_i h_i sum_q G(y_jq - x_i),  v_j += ... dG/dn_y(x_i, y_jq)
//                (the quadrature points of element j are now the evaluation
//                points and the centroids the sources; weight w_j at the end)
//   correction   C^T, scattered with atomic adds
//   far field    the forward chain L2P . L2L . M2L . M2M . P2M reversed with
//                every factor transposed: L2P^T (leaf sums of the L2P rows),
//                L2L^T upward, M2L^T across, M2M^T downward, P2M^T (dot
//                products with the P2M rows).
#include <cub/cub.cuh>

#include "bem_common.cuh"
#include "bem_f32x2.cuh"

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename R>
struct AV4;
template <>
struct AV4<float> {
  typedef float4 T;
};
template <>
struct AV4<double> {
  typedef double4 T;
};

// h = conj(g) in octree order, stored in the density workspace (.x, .y)
template <typename Rin, typename V4>
__global__ void k_adj_prologue(int64_t nt, int nrhs, const int* __restrict__ perm, const Rin* __restrict__ g,
                               V4* dens) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nt) return;
  int64_t o = perm[s];
  for (int r = 0; r < nrhs; ++r) {
    int64_t io = 2 * ((int64_t)r * nt + o);
    V4 d;
    d.x = g[io];
    d.y = -g[io + 1];
    d.z = 0;
    d.w = 0;
    dens[(int64_t)r * nt + s] = d;
  }
}

template <typename Rout>
__global__ void k_adj_epilogue(int64_t nt, int nrhs, const int* __restrict__ perm, const double* __restrict__ wgt,
                               const Rout* __restrict__ g, const double4* __restrict__ uv, int half, Rout* gx,
                               Rout* gy) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nt) return;
  int64_t o = perm[s];
  double w = wgt[s];
  for (int r = 0; r < nrhs; ++r) {
    double4 a = uv[(int64_t)r * nt + s];
    int64_t io = 2 * ((int64_t)r * nt + o);
    if (gy) {
      gy[io] = (Rout)(w * a.x);
      gy[io + 1] = (Rout)(-w * a.y);
    }
    if (gx) {
      double re = -w * a.z, im = w * a.w;  // -conj(v)
      if (half) {
        re += 0.5 * (double)g[io];
        im += 0.5 * (double)g[io + 1];
      }
      gx[io] = (Rout)re;
      gx[io + 1] = (Rout)im;
    }
  }
}

// contribution of the source centroid x (complex weight h) at one quadrature
// point y of an element with normal n:  u += h e^{ikr}/r,
// v += h (ikr - 1) e^{ikr}/r^3 (y - x).n   (dx = y - x)
template <typename R>
__device__ __forceinline__ void adj_point(R dx, R dy, R dz, R nx, R ny, R nz, R k, R hre, R him, R& ure, R& uim,
                                          R& vre, R& vim) {
  R r2 = dx * dx + dy * dy + dz * dz;
  R rinv, sn, cs;
  if (sizeof(R) == 4) {
    float ri = rsqrtf((float)r2);
    float s_, c_;
    __sincosf((float)k * (float)r2 * ri, &s_, &c_);
    rinv = (R)ri;
    sn = (R)s_;
    cs = (R)c_;
  } else {
    double rr = sqrt((double)r2);
    rinv = (R)(1.0 / rr);
    double s_, c_;
    sincos((double)k * rr, &s_, &c_);
    sn = (R)s_;
    cs = (R)c_;
  }
  R kr = k * r2 * rinv;
  R gre = rinv * cs, gim = rinv * sn;
  R f = (dx * nx + dy * ny + dz * nz) * rinv * rinv;
  R dre = f * (-gre - kr * gim), dim = f * (kr * gre - gim);
  ure += gre * hre - gim * him;
  uim += gre * him + gim * hre;
  vre += dre * hre - dim * him;
  vim += dre * him + dim * hre;
}

// near field, transposed: one warp per unit (leaf, 2^j elements j); lanes =
// element pairs x source slices, as in the forward kernel
#define ADJ_WARPS 4
template <typename R>
__global__ void __launch_bounds__(32 * ADJ_WARPS) k_p2p_adj(int nunits, int64_t nt, R k,
                                                            const int4* __restrict__ units,
                                                            const int* __restrict__ u_ptr,
                                                            const int* __restrict__ u_src,
                                                            const typename AV4<R>::T* __restrict__ u_shift,
                                                            const int* __restrict__ bstart,
                                                            const int* __restrict__ bend,
                                                            const typename AV4<R>::T* __restrict__ tgt,
                                                            const typename AV4<R>::T* __restrict__ src,
                                                            const typename AV4<R>::T* __restrict__ dens,
                                                            double4* __restrict__ uv) {
  typedef typename AV4<R>::T V4;
  int u = blockIdx.x * ADJ_WARPS + (threadIdx.x >> 5);
  if (u >= nunits) return;
  int lane = threadIdx.x & 31;
  int r = blockIdx.y;
  int4 U = units[u];
  int b = U.x, first = U.y, cnt = U.z;
  int np2 = (cnt + 1) >> 1;
  int pi = lane & (np2 - 1), split = lane / np2, nsplit = 32 / np2;
  bool two = pi + np2 < cnt;
  int ja = first + pi, jb = first + (two ? pi + np2 : pi);
  V4 qa[3], qb[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    qa[q] = src[3 * (int64_t)ja + q];
    qb[q] = src[3 * (int64_t)jb + q];
  }
  const V4* dr = dens + (int64_t)r * nt;
  const int ue = u_ptr[b + 1];
  R ua_re = 0, ua_im = 0, va_re = 0, va_im = 0, ub_re = 0, ub_im = 0, vb_re = 0, vb_im = 0;
  if constexpr (sizeof(R) == 4) {
    // packed: the lane's two elements a, b go through one f32x2 instruction
    // per operation; each source centroid and weight is broadcast once
    f32x2 px[3], py[3], pz[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      px[q] = pk2(qa[q].x, qb[q].x);
      py[q] = pk2(qa[q].y, qb[q].y);
      pz[q] = pk2(qa[q].z, qb[q].z);
    }
    const f32x2 pnx = pk2(qa[0].w, qb[0].w), pny = pk2(qa[1].w, qb[1].w), pnz = pk2(qa[2].w, qb[2].w);
    const f32x2 pk_k = pk2((float)k, (float)k);
    f32x2 u_re = pk2(0.f, 0.f), u_im = u_re, v_re = u_re, v_im = u_re;
    for (int ui = u_ptr[b]; ui < ue; ++ui) {
      const int sb = u_src[ui];
      const bool self = sb == b;  // own leaf: the pair of an element with itself is left out
      const V4 sh = u_shift[ui];  // centre(the other leaf) - centre(this leaf)
      const float sx = sh.x, sy = sh.y, sz = sh.z;
      int e1 = bend[sb];
      for (int e = bstart[sb] + split; e < e1; e += nsplit) {
        const V4 x = tgt[e];
        const V4 d = dr[e];
        const float nxx = -(x.x + sx), nxy = -(x.y + sy), nxz = -(x.z + sz);
        const f32x2 cx = pk2(nxx, nxx), cy = pk2(nxy, nxy), cz = pk2(nxz, nxz);
        const f32x2 hre = pk2(d.x, d.x), him = pk2(d.y, d.y), nhre = pk2(-d.x, -d.x), nhim = pk2(-d.y, -d.y);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const f32x2 dx = add2(px[q], cx), dy = add2(py[q], cy), dz = add2(pz[q], cz);
          const f32x2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
          float r2a, r2b;
          upk2(r2, r2a, r2b);
          f32x2 ri = pk2(rsqrtf(r2a), rsqrtf(r2b));
          if (self) ri = mul2(ri, pk2(e == ja ? 0.f : 1.f, e == jb ? 0.f : 1.f));
          const f32x2 kr = mul2(pk_k, mul2(r2, ri));
          float kra, krb, sa, ca, sb_, cb;
          upk2(kr, kra, krb);
          __sincosf(kra, &sa, &ca);  // |kr| stays small in the near field
          __sincosf(krb, &sb_, &cb);
          const f32x2 gre = mul2(ri, pk2(ca, cb)), gim = mul2(ri, pk2(sa, sb_));
          const f32x2 ngim = neg2(gim);
          const f32x2 f = mul2(fma2(dx, pnx, fma2(dy, pny, mul2(dz, pnz))), mul2(ri, ri));
          // (dre, dim) = f (ikr - 1) (gre + i gim)
          const f32x2 ndre = mul2(f, fma2(kr, gim, gre));      // -dre
          const f32x2 dim = mul2(f, fma2(kr, gre, ngim));
          u_re = fma2(gre, hre, fma2(ngim, him, u_re));
          u_im = fma2(gre, him, fma2(gim, hre, u_im));
          v_re = fma2(dim, nhim, fma2(ndre, nhre, v_re));
          v_im = fma2(dim, hre, fma2(ndre, nhim, v_im));
        }
      }
    }
    float lo, hi;
    upk2(u_re, lo, hi);
    ua_re = lo;
    ub_re = hi;
    upk2(u_im, lo, hi);
    ua_im = lo;
    ub_im = hi;
    upk2(v_re, lo, hi);
    va_re = lo;
    vb_re = hi;
    upk2(v_im, lo, hi);
    va_im = lo;
    vb_im = hi;
  } else
  for (int ui = u_ptr[b]; ui < ue; ++ui) {
    const int sb = u_src[ui];
    const bool self = sb == b;
    const V4 sh = u_shift[ui];
    const R sx = sh.x, sy = sh.y, sz = sh.z;
    int e1 = bend[sb];
    for (int e = bstart[sb] + split; e < e1; e += nsplit) {
      V4 x = tgt[e];
      V4 d = dr[e];
      R xx = x.x + sx, xy = x.y + sy, xz = x.z + sz;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (!(self && e == ja))
          adj_point<R>(qa[q].x - xx, qa[q].y - xy, qa[q].z - xz, qa[0].w, qa[1].w, qa[2].w, k, d.x, d.y, ua_re,
                       ua_im, va_re, va_im);
        if (!(self && e == jb))
          adj_point<R>(qb[q].x - xx, qb[q].y - xy, qb[q].z - xz, qb[0].w, qb[1].w, qb[2].w, k, d.x, d.y, ub_re,
                       ub_im, vb_re, vb_im);
      }
    }
  }
  for (int o = np2; o < 32; o <<= 1) {
    ua_re += __shfl_xor_sync(0xffffffffu, ua_re, o);
    ua_im += __shfl_xor_sync(0xffffffffu, ua_im, o);
    va_re += __shfl_xor_sync(0xffffffffu, va_re, o);
    va_im += __shfl_xor_sync(0xffffffffu, va_im, o);
    ub_re += __shfl_xor_sync(0xffffffffu, ub_re, o);
    ub_im += __shfl_xor_sync(0xffffffffu, ub_im, o);
    vb_re += __shfl_xor_sync(0xffffffffu, vb_re, o);
    vb_im += __shfl_xor_sync(0xffffffffu, vb_im, o);
  }
  if (split == 0) {
    uv[(int64_t)r * nt + ja] = make_double4(ua_re, ua_im, va_re, va_im);
    if (two) uv[(int64_t)r * nt + jb] = make_double4(ub_re, ub_im, vb_re, vb_im);
  }
}

// direct (all pairs), transposed: one element per thread, every centroid a source
template <typename R>
__global__ void __launch_bounds__(128) k_p2p_adj_direct(int64_t nt, R k, const typename AV4<R>::T* __restrict__ tgt,
                                                       const typename AV4<R>::T* __restrict__ src,
                                                       const typename AV4<R>::T* __restrict__ dens,
                                                       double4* __restrict__ uv) {
  typedef typename AV4<R>::T V4;
  __shared__ V4 s_x[128], s_h[128];
  int r = blockIdx.y;
  int64_t j = blockIdx.x * (int64_t)128 + threadIdx.x;
  const V4* dr = dens + (int64_t)r * nt;
  V4 q[3];
  int64_t jj = j < nt ? j : 0;
  for (int a = 0; a < 3; ++a) q[a] = src[3 * jj + a];
  double u0 = 0, u1 = 0, v0 = 0, v1 = 0;
  for (int64_t e0 = 0; e0 < nt; e0 += 128) {
    int ne = (int)min((int64_t)128, nt - e0);
    __syncthreads();
    if (threadIdx.x < ne) {
      s_x[threadIdx.x] = tgt[e0 + threadIdx.x];
      s_h[threadIdx.x] = dr[e0 + threadIdx.x];
    }
    __syncthreads();
    R ure = 0, uim = 0, vre = 0, vim = 0;
    for (int e = 0; e < ne; ++e) {
      if (e0 + e == j) continue;  // the self term comes whole from the correction
      V4 x = s_x[e], h = s_h[e];
      for (int a = 0; a < 3; ++a)
        adj_point<R>(q[a].x - x.x, q[a].y - x.y, q[a].z - x.z, q[0].w, q[1].w, q[2].w, k, h.x, h.y, ure, uim, vre,
                     vim);
    }
    u0 += ure;
    u1 += uim;
    v0 += vre;
    v1 += vim;
  }
  if (j < nt) uv[(int64_t)r * nt + j] = make_double4(u0, u1, v0, v1);
}

// correction, transposed: warp per row i, entries scattered into their columns
// the correction's transpose by counting sort: entries per column, their
// offsets, then every entry scattered to its column (order within a column
// follows the atomics)
__global__ void k_corrT_count(int64_t nnz, const int* __restrict__ col, int* cnt) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < nnz) atomicAdd(&cnt[col[e]], 1);
}
template <typename V4>
__global__ void k_corrT_fill(int64_t nt, const int* __restrict__ ptr, const int* __restrict__ col,
                             const V4* __restrict__ val, const int* __restrict__ ptrT, int* fill, int* rowT,
                             V4* valT) {
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= nt) return;
  for (int e = ptr[i] + lane; e < ptr[i + 1]; e += 32) {
    const int j = col[e];
    const int pos = ptrT[j] + atomicAdd(&fill[j], 1);
    rowT[pos] = (int)i;
    valT[pos] = val[e];
  }
}

// uv_j += sum_i C_ij h_i through the transpose: one warp per column j, the
// value and row loads of two entries per lane issued before their gathers,
// accumulated in the operator's precision
template <typename V4, typename R>
__global__ void k_corr_adj(int64_t nt, const int* __restrict__ ptrT, const int* __restrict__ rowT,
                           const V4* __restrict__ valT, const V4* __restrict__ dens, double4* __restrict__ uv) {
  const int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.y;
  if (j >= nt) return;
  const V4* dr = dens + (int64_t)r * nt;
  R ur = 0, ui = 0, vr = 0, vi = 0;
  const int e1 = ptrT[j + 1];
  for (int eb = ptrT[j] + lane; eb < e1; eb += 64) {
    V4 c[2];
    int ri[2];
#pragma unroll
    for (int u = 0; u < 2; ++u)
      if (eb + 32 * u < e1) {
        c[u] = valT[eb + 32 * u];
        ri[u] = rowT[eb + 32 * u];
      }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (eb + 32 * u >= e1) break;
      const V4 h = dr[ri[u]];
      ur += c[u].x * h.x - c[u].y * h.y;
      ui += c[u].x * h.y + c[u].y * h.x;
      vr += c[u].z * h.x - c[u].w * h.y;
      vi += c[u].z * h.y + c[u].w * h.x;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    ur += __shfl_xor_sync(0xffffffffu, ur, o);
    ui += __shfl_xor_sync(0xffffffffu, ui, o);
    vr += __shfl_xor_sync(0xffffffffu, vr, o);
    vi += __shfl_xor_sync(0xffffffffu, vi, o);
  }
  if (lane == 0) {
    double4* t = uv + (int64_t)r * nt + j;
    double4 a = *t;
    a.x += (double)ur;
    a.y += (double)ui;
    a.z += (double)vr;
    a.w += (double)vi;
    *t = a;
  }
}

template <typename V4>
static int build_corr_transpose(bem_handle* h, cudaStream_t s) {
  const int64_t nt = h->nt, nnz = h->corr_nnz;
  BEM_TRY(bem_alloc(h, &h->corrT_ptr, nt + 1));
  int* rowT;
  V4* valT;
  BEM_TRY(bem_alloc(h, &rowT, std::max<int64_t>(nnz, 1)));
  BEM_TRY(bem_alloc(h, &valT, std::max<int64_t>(nnz, 1)));
  h->corrT_row = rowT;
  h->corrT_val = valT;
  int *cnt = nullptr, *fill = nullptr;
  void* tmp = nullptr;
  BEM_CUDA(cudaMallocAsync((void**)&cnt, (nt + 1) * sizeof(int), s));
  BEM_CUDA(cudaMallocAsync((void**)&fill, nt * sizeof(int), s));
  BEM_CUDA(cudaMemsetAsync(cnt, 0, (nt + 1) * sizeof(int), s));
  BEM_CUDA(cudaMemsetAsync(fill, 0, nt * sizeof(int), s));
  if (nnz > 0) k_corrT_count<<<nblk(nnz, 256), 256, 0, s>>>(nnz, h->corr_col, cnt);
  size_t tb = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, tb, cnt, h->corrT_ptr, (int)nt + 1, s);
  BEM_CUDA(cudaMallocAsync(&tmp, tb, s));
  BEM_CUDA(cub::DeviceScan::ExclusiveSum(tmp, tb, cnt, h->corrT_ptr, (int)nt + 1, s));
  k_corrT_fill<V4><<<nblk(nt * 32, 256), 256, 0, s>>>(nt, h->corr_ptr, h->corr_col, (const V4*)h->corr_val,
                                                      h->corrT_ptr, fill, rowT, valT);
  BEM_CUDA(cudaGetLastError());
  cudaFreeAsync(tmp, s);
  cudaFreeAsync(cnt, s);
  cudaFreeAsync(fill, s);
  return BEM_OK;
}

int bem_build_corr_transpose(bem_handle* h, cudaStream_t s) {
  if (h->corrT_ptr) return BEM_OK;
  if (bem_is_fp64(h)) return build_corr_transpose<double4>(h, s);
  return build_corr_transpose<float4>(h, s);
}

// L2P^T: Lambda_b = sum_{i in b} rows_r[i] h_i  (leaf level)
template <typename R>
__global__ void k_l2p_t(int nleaf, const int* __restrict__ leafbox, int64_t nt, int P, const int* __restrict__ bstart,
                        const int* __restrict__ bend, const int64_t* __restrict__ row_off,
                        const R* __restrict__ rows_r, const typename AV4<R>::T* __restrict__ dens, int64_t exp_base,
                        int64_t exp_stride, R* __restrict__ Lam) {
  typedef typename AV4<R>::T V4;
  int b = leafbox[blockIdx.x], r = blockIdx.y;
  const V4* dr = dens + (int64_t)r * nt;
  const int64_t rb = row_off[bstart[b]], Pe = (P + 1) & ~1;  // the leaf's rows follow each other
  for (int e = threadIdx.x; e < P; e += blockDim.x) {
    R are = 0, aim = 0;
    for (int i = bstart[b]; i < bend[b]; ++i) {
      const R* row = rows_r + 2 * (rb + (i - bstart[b]) * Pe);
      R xr = row[2 * e], xi = row[2 * e + 1];
      V4 h = dr[i];
      are += xr * h.x - xi * h.y;
      aim += xr * h.y + xi * h.x;
    }
    R* out = Lam + 2 * ((int64_t)r * exp_stride + exp_base + (int64_t)b * P + e);
    out[0] = are;
    out[1] = aim;
  }
}

// P2M^T: u_j += a_j . Mu_b, v_j += b_j . Mu_b   (warp per element, leaf level)
template <typename R>
__global__ void k_p2m_t(int64_t nt, LevTab lt, const int* __restrict__ leaf_of,
                        const unsigned char* __restrict__ leaf_lev, const int64_t* __restrict__ row_off,
                        const R* __restrict__ rows_ab, const R* __restrict__ Mu, int64_t exp_stride,
                        double4* __restrict__ uv) {
  int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  int r = blockIdx.y;
  if (j >= nt) return;
  int b = leaf_of[j];
  const int lvl = leaf_lev[j];
  const int P = lt.P[lvl];  // 0 above level 2: no multipole
  const R* ab = rows_ab + 4 * row_off[j];
  const R* M = Mu + 2 * ((int64_t)r * exp_stride + lt.base[lvl] + (int64_t)b * P);
  R ure = 0, uim = 0, vre = 0, vim = 0;
  for (int e = lane; e < P; e += 32) {
    R mr = M[2 * e], mi = M[2 * e + 1];
    R ar = ab[2 * e], ai = ab[2 * e + 1], br = ab[2 * (P + e)], bi = ab[2 * (P + e) + 1];
    ure += ar * mr - ai * mi;
    uim += ar * mi + ai * mr;
    vre += br * mr - bi * mi;
    vim += br * mi + bi * mr;
  }
  for (int o = 16; o > 0; o >>= 1) {
    ure += __shfl_xor_sync(0xffffffffu, ure, o);
    uim += __shfl_xor_sync(0xffffffffu, uim, o);
    vre += __shfl_xor_sync(0xffffffffu, vre, o);
    vim += __shfl_xor_sync(0xffffffffu, vim, o);
  }
  if (lane == 0) {
    double4* t = uv + (int64_t)r * nt + j;
    double4 a = *t;
    a.x += ure;
    a.y += uim;
    a.z += vre;
    a.w += vim;
    *t = a;
  }
}

template <typename R>
static int adjoint_impl(bem_handle* h, int nrhs, cudaStream_t s) {
  typedef typename AV4<R>::T V4;
  int64_t nt = h->nt;
  const V4* dens = (const V4*)h->dens;
  const V4* tgt = (const V4*)(sizeof(R) == 4 ? (const void*)h->tgt32 : (const void*)h->tgt64);
  const V4* src = (const V4*)(sizeof(R) == 4 ? (const void*)h->src32 : (const void*)h->src64);
  bool fmm = bem_is_fmm(h);
  int L = h->L;
  int pr = bem_prof_begin(h, s);
  if (fmm) {
    dim3 grid(nblk(h->n_p2p_units, ADJ_WARPS), nrhs);
    const V4* ush = (const V4*)(sizeof(R) == 4 ? (const void*)h->u_shift32 : (const void*)h->u_shift64);
    k_p2p_adj<R><<<grid, 32 * ADJ_WARPS, 0, s>>>(h->n_p2p_units, nt, (R)h->k, h->p2p_units, h->u_ptr, h->u_src, ush,
                                                 h->gl_start, h->gl_end, tgt, src, dens, h->uv);
  } else {
    dim3 grid(nblk(nt, 128), nrhs);
    k_p2p_adj_direct<R><<<grid, 128, 0, s>>>(nt, (R)h->k, tgt, src, dens, h->uv);
  }
  BEM_CUDA(cudaGetLastError());
  bem_prof_end(h, pr, 1, 1, s);
  pr = bem_prof_begin(h, s);
  {
    dim3 grid(nblk(nt * 32, 256), nrhs);
    k_corr_adj<V4, R><<<grid, 256, 0, s>>>(nt, h->corrT_ptr, h->corrT_row, (const V4*)h->corrT_val, dens, h->uv);
    BEM_CUDA(cudaGetLastError());
  }
  bem_prof_end(h, pr, 2, 1, s);
  if (!fmm || L < 2) return BEM_OK;
  size_t esz = 2 * sizeof(R);
  const LevTab lt = bem_levtab(h);
  pr = bem_prof_begin(h, s);
  BEM_CUDA(cudaMemsetAsync(h->Mexp, 0, esz * h->exp_total * nrhs, s));
  BEM_CUDA(cudaMemsetAsync(h->Lexp, 0, esz * h->exp_total * nrhs, s));
  int nl = 0;
  for (int l = 2; l <= L; ++l) {
    LevelInfo& lf = h->lev[l];
    if (lf.nleaf == 0) continue;
    dim3 grid(lf.nleaf, nrhs);
    k_l2p_t<R><<<grid, 128, 0, s>>>(lf.nleaf, lf.leafbox, nt, lf.P, lf.start, lf.end, h->row_off,
                                    (const R*)h->l2p_rows, dens, lf.exp_base, h->exp_total, (R*)h->Lexp);
    BEM_CUDA(cudaGetLastError());
    ++nl;
  }
  BEM_TRY(bem_run_m2p_t(h, nrhs, dens, h->Mexp, s, &nl));  // W-lists: target weights into the multipoles
  bem_prof_end(h, pr, 7, nl, s);
  nl = 0;
  pr = bem_prof_begin(h, s);
  for (int l = L - 1; l >= 2; --l) BEM_TRY(bem_run_grouped(h, h->l2l_T[l], h->Lexp, h->Lexp, nrhs, s, &nl));
  bem_prof_end(h, pr, 6, nl, s);
  nl = 0;
  pr = bem_prof_begin(h, s);
  for (int l = 2; l <= L; ++l) BEM_TRY(bem_run_grouped(h, h->m2l_T[l], h->Lexp, h->Mexp, nrhs, s, &nl));
  BEM_TRY(bem_run_p2l_t(h, nrhs, h->Lexp, h->uv, s, &nl));  // X-lists: local weights back to the sources
  bem_prof_end(h, pr, 5, nl, s);
  nl = 0;
  pr = bem_prof_begin(h, s);
  for (int l = 2; l < L; ++l) BEM_TRY(bem_run_grouped(h, h->m2m_T[l], h->Mexp, h->Mexp, nrhs, s, &nl));
  bem_prof_end(h, pr, 4, nl, s);
  pr = bem_prof_begin(h, s);
  {
    dim3 grid(nblk(nt * 32, 256), nrhs);
    k_p2m_t<R><<<grid, 256, 0, s>>>(nt, lt, h->leaf_of, h->leaf_lev, h->row_off, (const R*)h->p2m_rows,
                                    (const R*)h->Mexp, h->exp_total, h->uv);
    BEM_CUDA(cudaGetLastError());
  }
  bem_prof_end(h, pr, 3, 1, s);
  return BEM_OK;
}

int bem_adjoint_sorted(bem_handle* h, int nrhs, int dtype, const void* g, void* gx, void* gy, int half,
                       cudaStream_t s) {
  BEM_TRY(bem_build_adjoint(h, s));
  int64_t nt = h->nt;
  unsigned gb = nblk(nt, 256);
  bool f64 = bem_is_fp64(h);
  if (dtype == BEM_C128) {
    if (f64)
      k_adj_prologue<double, double4><<<gb, 256, 0, s>>>(nt, nrhs, h->perm, (const double*)g, (double4*)h->dens);
    else
      k_adj_prologue<double, float4><<<gb, 256, 0, s>>>(nt, nrhs, h->perm, (const double*)g, (float4*)h->dens);
  } else {
    if (f64)
      k_adj_prologue<float, double4><<<gb, 256, 0, s>>>(nt, nrhs, h->perm, (const float*)g, (double4*)h->dens);
    else
      k_adj_prologue<float, float4><<<gb, 256, 0, s>>>(nt, nrhs, h->perm, (const float*)g, (float4*)h->dens);
  }
  BEM_CUDA(cudaGetLastError());
  if (f64)
    BEM_TRY(adjoint_impl<double>(h, nrhs, s));
  else
    BEM_TRY(adjoint_impl<float>(h, nrhs, s));
  if (dtype == BEM_C128)
    k_adj_epilogue<double><<<gb, 256, 0, s>>>(nt, nrhs, h->perm, h->wgt, (const double*)g, h->uv, half, (double*)gx,
                                              (double*)gy);
  else
    k_adj_epilogue<float><<<gb, 256, 0, s>>>(nt, nrhs, h->perm, h->wgt, (const float*)g, h->uv, half, (float*)gx,
                                             (float*)gy);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}
