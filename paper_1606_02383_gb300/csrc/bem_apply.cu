// bem_apply.cu -- the hot path: z = (1/2 I - D) x + S y  (Section 2.3, step 2(c)).
//
// Stages of one apply (on the caller's stream, except the far field, which
// runs on the handle's high-priority stream beside the correction):
//   prologue  : gather x, y into octree order, weighted by w_j = A_j/(12 pi)
//   P2P       : regular-rule near field, leaf box against its 27 colleagues,
//               FP32 (range-reduced sincos) or FP64
//   correction: CSR SpMV with the FP64-built near-singular / self corrections
//   P2M       : leaf multipoles from the stored per-element rows (HBM stream)
//   M2M, M2L, L2L : one grouped kernel, gather -> dense complex tile GEMM with
//               the translation matrix of the group -> scatter-add
//   L2P       : far field at the centroids from the stored per-element rows
//   epilogue  : z = 1/2 x + near + far, back to the caller's order and dtype
#include <algorithm>
#include <type_traits>

#include "bem_common.cuh"
#include "bem_tree_walk.cuh"
#include "bem_f32x2.cuh"
#include "bem_rules.cuh"

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename R>
struct V4of;
template <>
struct V4of<float> {
  typedef float4 T;
};
template <>
struct V4of<double> {
  typedef double4 T;
};

// ---------------------------------------------------------------- prologue --
template <typename Rin, typename V4>
__global__ void k_prologue(int64_t nt, int nrhs, const int* __restrict__ perm, const double* __restrict__ wgt,
                           const Rin* __restrict__ x, const Rin* __restrict__ y, V4* dens) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nt) return;
  int64_t o = perm[s];
  double w = wgt[s];
  for (int r = 0; r < nrhs; ++r) {
    int64_t io = 2 * ((int64_t)r * nt + o);
    V4 d;
    d.x = y ? (w * (double)y[io]) : 0.0;
    d.y = y ? (w * (double)y[io + 1]) : 0.0;
    d.z = x ? (w * (double)x[io]) : 0.0;
    d.w = x ? (w * (double)x[io + 1]) : 0.0;
    dens[(int64_t)r * nt + s] = d;
  }
}

// ---------------------------------------------------------------- epilogue --
template <typename Rout, typename Rin>
__global__ void k_epilogue(int64_t nt, int nrhs, const int* __restrict__ perm, const Rin* __restrict__ x, int half,
                           const double* __restrict__ zn, const double* __restrict__ zfar, Rout* z) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nt) return;
  int64_t o = perm[s];
  for (int r = 0; r < nrhs; ++r) {
    int64_t is = 2 * ((int64_t)r * nt + s), io = 2 * ((int64_t)r * nt + o);
    double re = zn[is], im = zn[is + 1];
    if (zfar) {
      re += zfar[is];
      im += zfar[is + 1];
    }
    if (half && x) {
      re += 0.5 * (double)x[io];
      im += 0.5 * (double)x[io + 1];
    }
    z[io] = (Rout)re;
    z[io + 1] = (Rout)im;
  }
}

// ------------------------------------------------------------- P2P (FMM) --
// One point of the combined regular-rule kernel.  With g = exp(ikr)/r,
// f = (y-x).n / r^2, sigma = w y and tau = w x (w = A/(12 pi)), the S and D
// contributions of the point are g sigma - (ikr - 1) g f tau
// = g [sigma + u - i kr u] with u = f tau.
__device__ __forceinline__ void p2p_eval(float dx, float dy, float dz, float nx, float ny, float nz, float k,
                                         float4 d, float& are, float& aim) {
  float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  float rinv = rsqrtf(r2);
  float kr = k * (r2 * rinv);
  float sn, cs;
  __sincosf(kr, &sn, &cs);  // |kr| stays small in the near field (phase error ~4e-8 kr)
  float f = fmaf(dx, nx, fmaf(dy, ny, dz * nz)) * (rinv * rinv);
  float ur = f * d.z, ui = f * d.w;
  float vr = fmaf(kr, ui, d.x + ur), vi = fmaf(-kr, ur, d.y + ui);
  float gre = rinv * cs, gim = rinv * sn;
  are = fmaf(gre, vr, fmaf(-gim, vi, are));
  aim = fmaf(gre, vi, fmaf(gim, vr, aim));
}
__device__ __forceinline__ void p2p_eval(double dx, double dy, double dz, double nx, double ny, double nz, double k,
                                         double4 d, double& are, double& aim) {
  double r2 = dx * dx + dy * dy + dz * dz;
  double r = sqrt(r2), rinv = 1.0 / r;
  double kr = k * r;
  double sn, cs;
  sincos(kr, &sn, &cs);
  double f = (dx * nx + dy * ny + dz * nz) * (rinv * rinv);
  double ur = f * d.z, ui = f * d.w;
  double vr = kr * ui + (d.x + ur), vi = -kr * ur + (d.y + ui);
  double gre = rinv * cs, gim = rinv * sn;
  are += gre * vr - gim * vi;
  aim += gre * vi + gim * vr;
}

// The point kernel of p2p_eval for two targets at once (packed pairs), split
// into the part every right-hand side shares (g = exp(ikr)/r, f and kr f) and
// the per-density update.  nt = (-t_a, -t_b) per axis; n as broadcast pairs;
// k2 = (k, k).
struct P2PPoint {
  f32x2 gre, gim, ngim, f, fk, nfk;
};
__device__ __forceinline__ P2PPoint p2p_point_pair(float qx, float qy, float qz, f32x2 ntx, f32x2 nty, f32x2 ntz,
                                                   f32x2 nx, f32x2 ny, f32x2 nz, f32x2 k2) {
  P2PPoint g;
  f32x2 dx = add2(pk2(qx, qx), ntx), dy = add2(pk2(qy, qy), nty), dz = add2(pk2(qz, qz), ntz);
  f32x2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
  float r2a, r2b;
  upk2(r2, r2a, r2b);
  f32x2 ri = pk2(rsqrtf(r2a), rsqrtf(r2b));
  f32x2 kr = mul2(k2, mul2(r2, ri));
  float kra, krb, sa, ca, sb, cb;
  upk2(kr, kra, krb);
  __sincosf(kra, &sa, &ca);  // |kr| stays small in the near field (phase error ~4e-8 kr)
  __sincosf(krb, &sb, &cb);
  g.f = mul2(fma2(dx, nx, fma2(dy, ny, mul2(dz, nz))), mul2(ri, ri));
  g.fk = mul2(g.f, kr);
  g.nfk = neg2(g.fk);
  g.gre = mul2(ri, pk2(ca, cb));
  g.gim = mul2(ri, pk2(sa, sb));
  g.ngim = neg2(g.gim);
  return g;
}
// a += g [sigma + u - i kr u], u = f tau, for the density d = (sigma, tau)
__device__ __forceinline__ void p2p_acc_pair(const P2PPoint& g, float4 d, f32x2& are, f32x2& aim) {
  f32x2 sre = pk2(d.x, d.x), sim = pk2(d.y, d.y), tre = pk2(d.z, d.z), tim = pk2(d.w, d.w);
  f32x2 vr = fma2(g.fk, tim, fma2(g.f, tre, sre));
  f32x2 vi = fma2(g.nfk, tre, fma2(g.f, tim, sim));
  are = fma2(g.gre, vr, fma2(g.ngim, vi, are));
  aim = fma2(g.gre, vi, fma2(g.gim, vr, aim));
}

// The contribution of element e to its own centroid t, computed with the
// operations of p2p_point_pair and p2p_acc_pair on one half of a pair (the
// packed instructions round each half like the scalar ones), both in the
// element's own leaf frame.
__device__ __forceinline__ void p2p_self_pair(float4 t, const float4* __restrict__ q, float4 d, float k, float& re,
                                              float& im) {
  const float4 q0 = q[0], q1 = q[1], q2 = q[2];
  const float nx = q0.w, ny = q1.w, nz = q2.w;
  const float ntx = 0.f - t.x, nty = 0.f - t.y, ntz = 0.f - t.z;
  re = im = 0.f;
  const float4 pts[3] = {q0, q1, q2};
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const float dx = pts[p].x + ntx, dy = pts[p].y + nty, dz = pts[p].z + ntz;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float ri = rsqrtf(r2);
    const float kr = k * (r2 * ri);
    float sn, cs;
    __sincosf(kr, &sn, &cs);
    const float f = fmaf(dx, nx, fmaf(dy, ny, dz * nz)) * (ri * ri);
    const float fk = f * kr;
    const float gre = ri * cs, gim = ri * sn;
    const float vr = fmaf(fk, d.w, fmaf(f, d.z, d.x));
    const float vi = fmaf(-fk, d.z, fmaf(f, d.w, d.y));
    re = fmaf(gre, vr, fmaf(-gim, vi, re));
    im = fmaf(gre, vi, fmaf(gim, vr, im));
  }
}

// One warp per work unit (leaf, 2^j consecutive targets, j <= 6).  The
// 32 lanes are np2 = ceil(count/2) target pairs times 32/np2 source slices;
// every lane owns two targets and walks its slice of the elements of the
// leaf's near list (every leaf that touches it, on any level; elements stored
// relative to their own leaf centre, shifted into the target leaf's frame on
// load), evaluating 6 points per element.  Slices are
// summed with an xor-shuffle butterfly; no shared memory and no barriers.
// Units are sorted by cost, largest first, so the tail of the grid is short.
#define P2P_WARPS 4
#define P2P_NR_MAX 4  // right-hand sides per FP32 P2P warp
// FP32: NR right-hand sides r0 + NR blockIdx.y + [0, NR) per warp, sharing
// the kernel values of every point (packed f32x2 arithmetic, two targets per
// lane).
// The end of a unit: take the self pair back out, sum the slices, write
template <int NR>
__device__ __forceinline__ void p2p_finish32(int r, int64_t nt, float k, int tfirst, int pi, int np2, int split,
                                             bool two, float4 ta, float4 tb, const float4* __restrict__ src,
                                             const float4* __restrict__ dr, f32x2 (&are)[NR], f32x2 (&aim)[NR],
                                             double* __restrict__ zn) {
  // The pair of a target with itself went through the loop (its own leaf is
  // in its near list); the near-singular correction carries the whole exact
  // self term, so the lane that writes the result takes it out again: the
  // same operations on the same values (FP32 rounding and all), so the FP32
  // cancellation of (y - x).n on the element's own plane leaves no trace.
  if (split == 0) {
    const int ia = tfirst + pi;
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      float ar, ai, br = 0.f, bi = 0.f;
      p2p_self_pair(ta, src + 3 * (int64_t)ia, dr[(int64_t)j * nt + ia], k, ar, ai);
      if (two) p2p_self_pair(tb, src + 3 * (int64_t)(ia + np2), dr[(int64_t)j * nt + ia + np2], k, br, bi);
      are[j] = sub2(are[j], pk2(ar, br));
      aim[j] = sub2(aim[j], pk2(ai, bi));
    }
  }
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    float a_re, b_re, a_im, b_im;
    upk2(are[j], a_re, b_re);
    upk2(aim[j], a_im, b_im);
    for (int o = np2; o < 32; o <<= 1) {
      a_re += __shfl_xor_sync(0xffffffffu, a_re, o);
      a_im += __shfl_xor_sync(0xffffffffu, a_im, o);
      b_re += __shfl_xor_sync(0xffffffffu, b_re, o);
      b_im += __shfl_xor_sync(0xffffffffu, b_im, o);
    }
    if (split == 0) {
      int64_t o = 2 * ((int64_t)(r + j) * nt + tfirst + pi);
      zn[o] = (double)a_re;
      zn[o + 1] = (double)a_im;
      if (two) {
        zn[o + 2 * np2] = (double)b_re;
        zn[o + 2 * np2 + 1] = (double)b_im;
      }
    }
  }
}

// one work unit u of the FP32 near field for right-hand sides r .. r + NR - 1
template <int NR>
__device__ __forceinline__ void p2p_unit32(int u, int r, int64_t nt, float k, const int4* __restrict__ units,
                                           const int* __restrict__ u_ptr, const int* __restrict__ u_src,
                                           const float4* __restrict__ u_shift, const int* __restrict__ bstart,
                                           const int* __restrict__ bend, const float4* __restrict__ tgt,
                                           const float4* __restrict__ src, const float4* __restrict__ dens,
                                           double* __restrict__ zn) {
  int lane = threadIdx.x & 31;
  int4 U = units[u];
  int b = U.x, tfirst = U.y, cnt = U.z;
  int np2 = (cnt + 1) >> 1;  // power of two
  int pi = lane & (np2 - 1), split = lane / np2, nsplit = 32 / np2;
  bool two = pi + np2 < cnt;
  float4 ta = tgt[tfirst + pi];
  float4 tb = tgt[tfirst + (two ? pi + np2 : pi)];
  const float4* dr = dens + (int64_t)r * nt;
  f32x2 are[NR], aim[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) are[j] = aim[j] = pk2(0.f, 0.f);
  const f32x2 pk_k = pk2(k, k);
  const int ue = u_ptr[b + 1];
  for (int ui = u_ptr[b]; ui < ue; ++ui) {
    const int sb = u_src[ui];
    const float4 sh = u_shift[ui];  // centre(source leaf) - centre(target leaf)
    const float sx = sh.x, sy = sh.y, sz = sh.z;
    // targets in the source box's frame, negated
    f32x2 ntx = pk2(sx - ta.x, sx - tb.x), nty = pk2(sy - ta.y, sy - tb.y), ntz = pk2(sz - ta.z, sz - tb.z);
    int e1 = bend[sb];
    for (int e = bstart[sb] + split; e < e1; e += nsplit) {
      float4 q0 = src[3 * (int64_t)e], q1 = src[3 * (int64_t)e + 1], q2 = src[3 * (int64_t)e + 2];
      float4 d[NR];
#pragma unroll
      for (int j = 0; j < NR; ++j) d[j] = dr[(int64_t)j * nt + e];
      f32x2 nx = pk2(q0.w, q0.w), ny = pk2(q1.w, q1.w), nz = pk2(q2.w, q2.w);
      P2PPoint g = p2p_point_pair(q0.x, q0.y, q0.z, ntx, nty, ntz, nx, ny, nz, pk_k);
#pragma unroll
      for (int j = 0; j < NR; ++j) p2p_acc_pair(g, d[j], are[j], aim[j]);
      g = p2p_point_pair(q1.x, q1.y, q1.z, ntx, nty, ntz, nx, ny, nz, pk_k);
#pragma unroll
      for (int j = 0; j < NR; ++j) p2p_acc_pair(g, d[j], are[j], aim[j]);
      g = p2p_point_pair(q2.x, q2.y, q2.z, ntx, nty, ntz, nx, ny, nz, pk_k);
#pragma unroll
      for (int j = 0; j < NR; ++j) p2p_acc_pair(g, d[j], are[j], aim[j]);
    }
  }
  p2p_finish32<NR>(r, nt, k, tfirst, pi, np2, split, two, ta, tb, src, dr, are, aim, zn);
}

template <int NR>
__global__ void __launch_bounds__(32 * P2P_WARPS) k_p2p_fmm32(int nunits, int64_t nt, int r0, float k,
                                                              const int4* __restrict__ units,
                                                              const int* __restrict__ u_ptr,
                                                              const int* __restrict__ u_src,
                                                              const float4* __restrict__ u_shift,
                                                              const int* __restrict__ bstart,
                                                              const int* __restrict__ bend,
                                                              const float4* __restrict__ tgt,
                                                              const float4* __restrict__ src,
                                                              const float4* __restrict__ dens,
                                                              double* __restrict__ zn) {
  const int u = blockIdx.x * P2P_WARPS + (threadIdx.x >> 5);
  if (u >= nunits) return;
  p2p_unit32<NR>(u, r0 + blockIdx.y * NR, nt, k, units, u_ptr, u_src, u_shift, bstart, bend, tgt, src, dens, zn);
}

// The same unit with the near list's source elements staged in shared memory:
// the list's elements, leaf after leaf, are cut into chunks of 32; lane j of
// the warp copies element j of a chunk (its three points, its leaf's centre
// offset and its NR densities, 16-byte cp.async pieces) into one of the
// warp's two buffers, and the lanes evaluate the other buffer meanwhile, so
// the loads of chunk c + 1 are in flight while chunk c is summed.
#define P2P_CH 32
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
template <int NR>
__device__ __forceinline__ void p2p_unit32_staged(int u, int r, int64_t nt, float k, const int4* __restrict__ units,
                                                  const int* __restrict__ u_ptr, const int* __restrict__ u_src,
                                                  const float4* __restrict__ u_shift, const int* __restrict__ bstart,
                                                  const int* __restrict__ bend, const float4* __restrict__ tgt,
                                                  const float4* __restrict__ src, const float4* __restrict__ dens,
                                                  float4* buf, double* __restrict__ zn) {
  constexpr int REC = 4 + NR;  // q0, q1, q2, leaf offset, densities
  const int lane = threadIdx.x & 31;
  const int4 U = units[u];
  const int b = U.x, tfirst = U.y, cnt = U.z;
  const int np2 = (cnt + 1) >> 1;  // power of two
  const int pi = lane & (np2 - 1), split = lane / np2, nsplit = 32 / np2;
  const bool two = pi + np2 < cnt;
  const float4 ta = tgt[tfirst + pi];
  const float4 tb = tgt[tfirst + (two ? pi + np2 : pi)];
  const float4* dr = dens + (int64_t)r * nt;
  f32x2 are[NR], aim[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) are[j] = aim[j] = pk2(0.f, 0.f);
  const f32x2 pk_k = pk2(k, k);
  const int ub = u_ptr[b], ue = u_ptr[b + 1];
  // warp-uniform cursor: list entry cu, element ce (ce = bend of entry cu when done)
  int cu = ub, ce = ub < ue ? bstart[u_src[ub]] : 0;
  // stage the next chunk into buffer s; returns its element count
  auto fill = [&](int s) -> int {
    int li = cu, le = ce, rem = lane;
    bool found = false;
    while (li < ue) {
      const int e1 = bend[u_src[li]];
      if (le + rem < e1) {
        le += rem;
        found = true;
        break;
      }
      rem -= e1 - le;
      ++li;
      if (li < ue) le = bstart[u_src[li]];
    }
    if (found) {
      float4* rec = buf + (s * P2P_CH + lane) * REC;
      const float4* q = src + 3 * (int64_t)le;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_u32(rec + c)), "l"(q + c) : "memory");
      asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_u32(rec + 3)), "l"(u_shift + li)
                   : "memory");
#pragma unroll
      for (int j = 0; j < NR; ++j)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_u32(rec + 4 + j)),
                     "l"(dr + (int64_t)j * nt + le)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    const unsigned got = __ballot_sync(0xffffffffu, found);
    const int n = __popc(got);
    // advance the cursor past the chunk: the element after the last lane's
    if (n == P2P_CH) {
      int nli = __shfl_sync(0xffffffffu, li, 31), nle = __shfl_sync(0xffffffffu, le, 31) + 1;
      if (nle >= bend[u_src[nli]]) {
        ++nli;
        nle = nli < ue ? bstart[u_src[nli]] : 0;
      }
      cu = nli;
      ce = nle;
    } else {
      cu = ue;
    }
    return n;
  };
  // one cp.async group per chunk slot, empty once the list is exhausted, so
  // that "all but the newest group landed" always means "chunk c landed"
  int n0 = fill(0), n1 = 0;
  if (n0 == P2P_CH)
    n1 = fill(1);
  else
    asm volatile("cp.async.commit_group;" ::: "memory");
  for (int c = 0; n0 > 0; ++c) {
    // chunk c (buffer c & 1) has landed once only the next chunk's copies are pending
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncwarp();
    const float4* cb = buf + (c & 1) * P2P_CH * REC;
    for (int e = split; e < n0; e += nsplit) {
      const float4* rec = cb + e * REC;
      const float4 q0 = rec[0], q1 = rec[1], q2 = rec[2], sh = rec[3];
      float4 d[NR];
#pragma unroll
      for (int j = 0; j < NR; ++j) d[j] = rec[4 + j];
      const f32x2 ntx = pk2(sh.x - ta.x, sh.x - tb.x), nty = pk2(sh.y - ta.y, sh.y - tb.y),
                  ntz = pk2(sh.z - ta.z, sh.z - tb.z);
      const f32x2 nx = pk2(q0.w, q0.w), ny = pk2(q1.w, q1.w), nz = pk2(q2.w, q2.w);
      P2PPoint g = p2p_point_pair(q0.x, q0.y, q0.z, ntx, nty, ntz, nx, ny, nz, pk_k);
#pragma unroll
      for (int j = 0; j < NR; ++j) p2p_acc_pair(g, d[j], are[j], aim[j]);
      g = p2p_point_pair(q1.x, q1.y, q1.z, ntx, nty, ntz, nx, ny, nz, pk_k);
#pragma unroll
      for (int j = 0; j < NR; ++j) p2p_acc_pair(g, d[j], are[j], aim[j]);
      g = p2p_point_pair(q2.x, q2.y, q2.z, ntx, nty, ntz, nx, ny, nz, pk_k);
#pragma unroll
      for (int j = 0; j < NR; ++j) p2p_acc_pair(g, d[j], are[j], aim[j]);
    }
    __syncwarp();  // every lane is done with buffer c & 1 before it is refilled
    n0 = n1;
    if (n1 == P2P_CH) {
      n1 = fill(c & 1);  // chunk c + 2
    } else {
      n1 = 0;
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  p2p_finish32<NR>(r, nt, k, tfirst, pi, np2, split, two, ta, tb, src, dr, are, aim, zn);
}

template <int NR>
__global__ void __launch_bounds__(32 * P2P_WARPS) k_p2p_fmm32_s(int nunits, int64_t nt, int r0, float k,
                                                                const int4* __restrict__ units,
                                                                const int* __restrict__ u_ptr,
                                                                const int* __restrict__ u_src,
                                                                const float4* __restrict__ u_shift,
                                                                const int* __restrict__ bstart,
                                                                const int* __restrict__ bend,
                                                                const float4* __restrict__ tgt,
                                                                const float4* __restrict__ src,
                                                                const float4* __restrict__ dens,
                                                                double* __restrict__ zn) {
  extern __shared__ __align__(16) float4 p2p_stage[];
  const int warp = threadIdx.x >> 5;
  const int u = blockIdx.x * P2P_WARPS + warp;
  if (u >= nunits) return;
  p2p_unit32_staged<NR>(u, r0 + blockIdx.y * NR, nt, k, units, u_ptr, u_src, u_shift, bstart, bend, tgt, src, dens,
                        p2p_stage + warp * 2 * P2P_CH * (4 + NR), zn);
}

// The same work from a fixed number of resident CTAs: every warp takes the
// next unit (largest first) from a counter per right-hand-side chunk, so the
// near field can run with a few CTAs per SM and leave room on every SM for
// the far field's kernels, which run beside it on the far-field stream.
template <int NR>
__global__ void __launch_bounds__(32 * P2P_WARPS) k_p2p_fmm32_q(int nunits, int64_t nt, int r0, float k,
                                                                int* __restrict__ counter,
                                                                const int4* __restrict__ units,
                                                                const int* __restrict__ u_ptr,
                                                                const int* __restrict__ u_src,
                                                                const float4* __restrict__ u_shift,
                                                                const int* __restrict__ bstart,
                                                                const int* __restrict__ bend,
                                                                const float4* __restrict__ tgt,
                                                                const float4* __restrict__ src,
                                                                const float4* __restrict__ dens,
                                                                double* __restrict__ zn) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    int u = 0;
    if (lane == 0) u = atomicAdd(&counter[blockIdx.y], 1);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= nunits) return;
    p2p_unit32<NR>(u, r0 + blockIdx.y * NR, nt, k, units, u_ptr, u_src, u_shift, bstart, bend, tgt, src, dens, zn);
  }
}

// FP64: one right-hand side per warp (grid.y), scalar arithmetic.
__global__ void __launch_bounds__(32 * P2P_WARPS) k_p2p_fmm64(int nunits, int64_t nt, double k,
                                                              const int4* __restrict__ units,
                                                              const int* __restrict__ u_ptr,
                                                              const int* __restrict__ u_src,
                                                              const double4* __restrict__ u_shift,
                                                              const int* __restrict__ bstart,
                                                              const int* __restrict__ bend,
                                                              const double4* __restrict__ tgt,
                                                              const double4* __restrict__ src,
                                                              const double4* __restrict__ dens,
                                                              double* __restrict__ zn) {
  int u = blockIdx.x * P2P_WARPS + (threadIdx.x >> 5);
  if (u >= nunits) return;
  int lane = threadIdx.x & 31;
  int r = blockIdx.y;
  int4 U = units[u];
  int b = U.x, tfirst = U.y, cnt = U.z;
  int np2 = (cnt + 1) >> 1;  // power of two
  int pi = lane & (np2 - 1), split = lane / np2, nsplit = 32 / np2;
  bool two = pi + np2 < cnt;
  double4 ta = tgt[tfirst + pi];
  double4 tb = tgt[tfirst + (two ? pi + np2 : pi)];
  const double4* dr = dens + (int64_t)r * nt;
  double a_re = 0, a_im = 0, b_re = 0, b_im = 0;
  const int ia = tfirst + pi, ib = tfirst + (two ? pi + np2 : pi);
  const int ue = u_ptr[b + 1];
  for (int ui = u_ptr[b]; ui < ue; ++ui) {
    const int sb = u_src[ui];
    const bool self = sb == b;  // the target's own leaf: the pair of a target with itself is left out
    const double4 sh = u_shift[ui];  // centre(source leaf) - centre(target leaf)
    const double sx = sh.x, sy = sh.y, sz = sh.z;
    double ax = ta.x - sx, ay = ta.y - sy, az = ta.z - sz;  // targets in the source box's frame
    double bx_ = tb.x - sx, by_ = tb.y - sy, bz_ = tb.z - sz;
    int e1 = bend[sb];
    for (int e = bstart[sb] + split; e < e1; e += nsplit) {
      double4 q0 = src[3 * (int64_t)e], q1 = src[3 * (int64_t)e + 1], q2 = src[3 * (int64_t)e + 2];
      double4 d = dr[e];
      double nx = q0.w, ny = q1.w, nz = q2.w;
      if (!(self && e == ia)) {
        p2p_eval(q0.x - ax, q0.y - ay, q0.z - az, nx, ny, nz, k, d, a_re, a_im);
        p2p_eval(q1.x - ax, q1.y - ay, q1.z - az, nx, ny, nz, k, d, a_re, a_im);
        p2p_eval(q2.x - ax, q2.y - ay, q2.z - az, nx, ny, nz, k, d, a_re, a_im);
      }
      if (!(self && e == ib)) {
        p2p_eval(q0.x - bx_, q0.y - by_, q0.z - bz_, nx, ny, nz, k, d, b_re, b_im);
        p2p_eval(q1.x - bx_, q1.y - by_, q1.z - bz_, nx, ny, nz, k, d, b_re, b_im);
        p2p_eval(q2.x - bx_, q2.y - by_, q2.z - bz_, nx, ny, nz, k, d, b_re, b_im);
      }
    }
  }
  for (int o = np2; o < 32; o <<= 1) {
    a_re += __shfl_xor_sync(0xffffffffu, a_re, o);
    a_im += __shfl_xor_sync(0xffffffffu, a_im, o);
    b_re += __shfl_xor_sync(0xffffffffu, b_re, o);
    b_im += __shfl_xor_sync(0xffffffffu, b_im, o);
  }
  if (split == 0) {
    int64_t o = 2 * ((int64_t)r * nt + tfirst + pi);
    zn[o] = a_re;
    zn[o + 1] = a_im;
    if (two) {
      zn[o + 2 * np2] = b_re;
      zn[o + 2 * np2 + 1] = b_im;
    }
  }
}

// ----------------------------------------------------------- direct sums --
#define P2P_THREADS 128
// One target per thread; all sources streamed through shared memory.  FP32
// partial sums are flushed into FP64 accumulators after every tile.
template <typename R>
__global__ void __launch_bounds__(P2P_THREADS) k_p2p_direct(int64_t nt, R k, const typename V4of<R>::T* __restrict__ tgt,
                                                            const typename V4of<R>::T* __restrict__ src,
                                                            const typename V4of<R>::T* __restrict__ dens,
                                                            double* __restrict__ zn) {
  typedef typename V4of<R>::T V4;
  __shared__ V4 s_src[P2P_THREADS][3];
  __shared__ V4 s_den[P2P_THREADS];
  int r = blockIdx.y;
  int64_t i = blockIdx.x * (int64_t)P2P_THREADS + threadIdx.x;
  const V4* dr = dens + (int64_t)r * nt;
  V4 tg;
  if (i < nt) tg = tgt[i];
  else tg = tgt[0];
  double sre = 0.0, sim = 0.0;
  for (int64_t e0 = 0; e0 < nt; e0 += P2P_THREADS) {
    int ne = (int)min((int64_t)P2P_THREADS, nt - e0);
    __syncthreads();
    if (threadIdx.x < ne) {
      for (int q = 0; q < 3; ++q) s_src[threadIdx.x][q] = src[3 * (e0 + threadIdx.x) + q];
      s_den[threadIdx.x] = dr[e0 + threadIdx.x];
    }
    __syncthreads();
    R are = 0, aim = 0;
    for (int e = 0; e < ne; ++e) {
      if (e0 + e == i) continue;  // the self term comes whole from the correction
      V4 q0 = s_src[e][0], q1 = s_src[e][1], q2 = s_src[e][2];
      V4 dd = s_den[e];
      R nx = q0.w, ny = q1.w, nz = q2.w;
      p2p_eval(q0.x - tg.x, q0.y - tg.y, q0.z - tg.z, nx, ny, nz, k, dd, are, aim);
      p2p_eval(q1.x - tg.x, q1.y - tg.y, q1.z - tg.z, nx, ny, nz, k, dd, are, aim);
      p2p_eval(q2.x - tg.x, q2.y - tg.y, q2.z - tg.z, nx, ny, nz, k, dd, are, aim);
    }
    sre += (double)are;
    sim += (double)aim;
  }
  if (i < nt) {
    int64_t o = 2 * ((int64_t)r * nt + i);
    zn[o] = sre;
    zn[o + 1] = sim;
  }
}

// ------------------------------------------------- off-surface evaluation --
// u(p) = sum_j S(p, j) y_j - D(p, j) x_j at points p off the surface, with the
// entries' rules: R_L (L = 2 within 2 h_j, 1 within 4 h_j of the centroid),
// R_0 beyond.  One point per thread; all elements stream through shared
// memory, relative to the block's first point (subtracted in FP64 once per
// element and block), so that the R_0 sums run in the operator's precision.
// A pair within 4 h_j instead takes the refined rule from the FP64 geometry,
// relative to its point.  FP32 partial sums go into FP64 after every tile.
#define EV_THREADS 128
template <typename R>
__device__ __forceinline__ void eval_near(const double* X, int j, double k, const double* __restrict__ cent,
                                          const double* __restrict__ qpt, const double* __restrict__ nrm,
                                          const double* __restrict__ area, const double* __restrict__ hmax,
                                          const double* __restrict__ wgt, const typename V4of<R>::T& dd, R& are,
                                          R& aim) {
  Tri64 t;
  load_tri64(qpt, nrm, cent, area, hmax, j, t);
  const double c0 = t.c[0] - X[0], c1 = t.c[1] - X[1], c2 = t.c[2] - X[2];
  const double dist = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
  const int L = dist < 2.0 * t.h ? 2 : (dist < 4.0 * t.h ? 1 : 0);
  const double iw = 1.0 / wgt[j];
  if constexpr (sizeof(R) == 4) {
    Tri32 tf;
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) tf.v[a][c] = (float)(t.v[a][c] - X[c]);
    for (int c = 0; c < 3; ++c) tf.n[c] = (float)t.n[c];
    tf.area = (float)t.area;
    zf sv = cmk(0.f, 0.f), dv = sv;
    rule_refined32(tf, L, (float)k, sv, dv);
    const float w = (float)iw;
    const float yr = dd.x * w, yi = dd.y * w, xr = dd.z * w, xi = dd.w * w;
    are += sv.re * yr - sv.im * yi - (dv.re * xr - dv.im * xi);
    aim += sv.re * yi + sv.im * yr - (dv.re * xi + dv.im * xr);
  } else {
    zd sv = cmk(0.0, 0.0), dv = sv;
    rule_refined(X, t, L, k, sv, dv);
    const double yr = dd.x * iw, yi = dd.y * iw, xr = dd.z * iw, xi = dd.w * iw;
    are += sv.re * yr - sv.im * yi - (dv.re * xr - dv.im * xi);
    aim += sv.re * yi + sv.im * yr - (dv.re * xi + dv.im * xr);
  }
}

template <typename R, typename Rout>
__global__ void __launch_bounds__(EV_THREADS) k_eval_points(int64_t nt, int64_t np, double k,
                                                            const double* __restrict__ pts,
                                                            const double* __restrict__ cent,
                                                            const double* __restrict__ qpt,
                                                            const double* __restrict__ nrm,
                                                            const double* __restrict__ area,
                                                            const double* __restrict__ hmax,
                                                            const double* __restrict__ wgt,
                                                            const typename V4of<R>::T* __restrict__ dens,
                                                            int nc, int c0, Rout* __restrict__ out) {
  typedef typename V4of<R>::T V4;
  __shared__ V4 s_q[EV_THREADS][3];  // quadrature points relative to the origin, normal in .w
  __shared__ V4 s_c[EV_THREADS];     // centroid relative to the origin, (4 h)^2 in .w
  __shared__ V4 s_d[EV_THREADS];     // weighted densities (sigma, tau)
  const int r = blockIdx.y;
  const int64_t p0 = blockIdx.x * (int64_t)EV_THREADS, p = p0 + threadIdx.x;
  const bool live = p < np;
  const double o[3] = {pts[3 * p0], pts[3 * p0 + 1], pts[3 * p0 + 2]};
  const int64_t pp = live ? p : p0;
  const double X[3] = {pts[3 * pp], pts[3 * pp + 1], pts[3 * pp + 2]};
  const R tx = (R)(X[0] - o[0]), ty = (R)(X[1] - o[1]), tz = (R)(X[2] - o[2]);
  const V4* dr = dens + (int64_t)r * nt;
  const R kr = (R)k;
  double sre = 0.0, sim = 0.0;
  for (int64_t e0 = 0; e0 < nt; e0 += EV_THREADS) {
    const int ne = (int)min((int64_t)EV_THREADS, nt - e0);
    __syncthreads();
    if (threadIdx.x < ne) {
      const int64_t j = e0 + threadIdx.x;
      for (int q = 0; q < 3; ++q) {
        V4 v;
        v.x = (R)(qpt[9 * j + 3 * q] - o[0]);
        v.y = (R)(qpt[9 * j + 3 * q + 1] - o[1]);
        v.z = (R)(qpt[9 * j + 3 * q + 2] - o[2]);
        v.w = (R)nrm[3 * j + q];
        s_q[threadIdx.x][q] = v;
      }
      const double h4 = 4.0 * hmax[j];
      V4 c;
      c.x = (R)(cent[3 * j] - o[0]);
      c.y = (R)(cent[3 * j + 1] - o[1]);
      c.z = (R)(cent[3 * j + 2] - o[2]);
      c.w = (R)(h4 * h4);
      s_c[threadIdx.x] = c;
      s_d[threadIdx.x] = dr[j];
    }
    __syncthreads();
    R are = 0, aim = 0;
    for (int e = 0; e < ne; ++e) {
      const V4 c = s_c[e];
      const R cx = c.x - tx, cy = c.y - ty, cz = c.z - tz;
      const V4 dd = s_d[e];
      if (cx * cx + cy * cy + cz * cz < c.w) {
        eval_near<R>(X, (int)(e0 + e), k, cent, qpt, nrm, area, hmax, wgt, dd, are, aim);
        continue;
      }
      const V4 q0 = s_q[e][0], q1 = s_q[e][1], q2 = s_q[e][2];
      const R nx = q0.w, ny = q1.w, nz = q2.w;
      p2p_eval(q0.x - tx, q0.y - ty, q0.z - tz, nx, ny, nz, kr, dd, are, aim);
      p2p_eval(q1.x - tx, q1.y - ty, q1.z - tz, nx, ny, nz, kr, dd, are, aim);
      p2p_eval(q2.x - tx, q2.y - ty, q2.z - tz, nx, ny, nz, kr, dd, are, aim);
    }
    sre += (double)are;
    sim += (double)aim;
  }
  if (live) {
    out[2 * (((int64_t)r * np + p) * nc + c0)] = (Rout)sre;
    out[2 * (((int64_t)r * np + p) * nc + c0) + 1] = (Rout)sim;
  }
}

// Gradient with respect to the field point of one rule point's contribution:
// with d = y - x, F = exp(ikr)(ikr - 1)/r^3 and H = exp(ikr)(3 - 3ikr - k^2 r^2)/r^5,
//   grad S-term = -F d sigma,  grad D-term = -(H (d.n) d + F n) tau,
// so grad u += d (-F sigma + (d.n) H tau) + n F tau  (sigma, tau weighted as
// in the apply: they carry the point weight and 1/(4 pi)).  Accurate sincos:
// a field point may be far from the sources.
template <typename R>
__device__ __forceinline__ void grad_eval(R dx, R dy, R dz, R nx, R ny, R nz, R k, R sr, R si, R tr, R ti,
                                          R (&g)[6]) {
  const R r2 = dx * dx + dy * dy + dz * dz;
  const R r = sqrt(r2), ir = R(1) / r, ir2 = ir * ir;
  const R kr = k * r;
  R sn, cs;
  if constexpr (sizeof(R) == 4) sincosf(kr, &sn, &cs);
  else sincos(kr, &sn, &cs);
  const R ir3 = ir * ir2, ir5 = ir3 * ir2;
  const R fr = (-cs - kr * sn) * ir3, fi = (kr * cs - sn) * ir3;
  const R q = R(3) - kr * kr;
  const R hr = (cs * q + R(3) * kr * sn) * ir5, hi = (sn * q - R(3) * kr * cs) * ir5;
  const R dn = dx * nx + dy * ny + dz * nz;
  const R ar = -(fr * sr - fi * si) + dn * (hr * tr - hi * ti);
  const R ai = -(fr * si + fi * sr) + dn * (hr * ti + hi * tr);
  const R br = fr * tr - fi * ti, bi = fr * ti + fi * tr;
  g[0] += ar * dx + br * nx;
  g[1] += ai * dx + bi * nx;
  g[2] += ar * dy + br * ny;
  g[3] += ai * dy + bi * ny;
  g[4] += ar * dz + br * nz;
  g[5] += ai * dz + bi * nz;
}

// the gradient contribution of element j under its refined rule, relative to X
template <typename R>
__device__ void grad_near(const double* X, int j, double k, const double* __restrict__ cent,
                          const double* __restrict__ qpt, const double* __restrict__ nrm,
                          const double* __restrict__ area, const double* __restrict__ hmax,
                          const typename V4of<R>::T& dd, R (&g)[6]) {
  Tri64 t;
  load_tri64(qpt, nrm, cent, area, hmax, j, t);
  const double c0 = t.c[0] - X[0], c1 = t.c[1] - X[1], c2 = t.c[2] - X[2];
  const double dist = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
  const int L = dist < 2.0 * t.h ? 2 : (dist < 4.0 * t.h ? 1 : 0);
  const int npieces = 1 << (2 * L);
  // each piece carries 1/4^L of the element's weight
  const R sc = R(1) / npieces;
  const R sr = dd.x * sc, si = dd.y * sc, tr = dd.z * sc, ti = dd.w * sc;
  const R nx = (R)t.n[0], ny = (R)t.n[1], nz = (R)t.n[2];
  for (int piece = 0; piece < npieces; ++piece) {
    R a[3], b[3], c[3];
    for (int e = 0; e < 3; ++e) {
      a[e] = (R)(t.v[0][e] - X[e]);
      b[e] = (R)(t.v[1][e] - X[e]);
      c[e] = (R)(t.v[2][e] - X[e]);
    }
    int code = piece;
    for (int lvl = 0; lvl < L; ++lvl) {
      const int child = code & 3;
      code >>= 2;
      R ab[3], bc[3], ca[3];
      for (int e = 0; e < 3; ++e) {
        ab[e] = R(0.5) * (a[e] + b[e]);
        bc[e] = R(0.5) * (b[e] + c[e]);
        ca[e] = R(0.5) * (c[e] + a[e]);
      }
      for (int e = 0; e < 3; ++e) {
        if (child == 0) {
          b[e] = ab[e];
          c[e] = ca[e];
        } else if (child == 1) {
          a[e] = ab[e];
          c[e] = bc[e];
        } else if (child == 2) {
          a[e] = ca[e];
          b[e] = bc[e];
        } else {
          a[e] = ab[e];
          b[e] = bc[e];
          c[e] = ca[e];
        }
      }
    }
    const R b0 = R(2) / R(3), b1 = R(1) / R(6);
    for (int q = 0; q < 3; ++q) {
      R y[3];
      for (int e = 0; e < 3; ++e)
        y[e] = (q == 0 ? b0 : b1) * a[e] + (q == 1 ? b0 : b1) * b[e] + (q == 2 ? b0 : b1) * c[e];
      grad_eval<R>(y[0], y[1], y[2], nx, ny, nz, (R)k, sr, si, tr, ti, g);
    }
  }
}

// grad u at points off the surface: as k_eval_points, three complex
// components per point, out [nrhs][np][3]
template <typename R, typename Rout>
__global__ void __launch_bounds__(EV_THREADS) k_eval_points_grad(int64_t nt, int64_t np, double k,
                                                                 const double* __restrict__ pts,
                                                                 const double* __restrict__ cent,
                                                                 const double* __restrict__ qpt,
                                                                 const double* __restrict__ nrm,
                                                                 const double* __restrict__ area,
                                                                 const double* __restrict__ hmax,
                                                                 const typename V4of<R>::T* __restrict__ dens,
                                                                 int nc, int c0, Rout* __restrict__ out) {
  typedef typename V4of<R>::T V4;
  __shared__ V4 s_q[EV_THREADS][3];
  __shared__ V4 s_c[EV_THREADS];
  __shared__ V4 s_d[EV_THREADS];
  const int r = blockIdx.y;
  const int64_t p0 = blockIdx.x * (int64_t)EV_THREADS, p = p0 + threadIdx.x;
  const bool live = p < np;
  const double o[3] = {pts[3 * p0], pts[3 * p0 + 1], pts[3 * p0 + 2]};
  const int64_t pp = live ? p : p0;
  const double X[3] = {pts[3 * pp], pts[3 * pp + 1], pts[3 * pp + 2]};
  const R tx = (R)(X[0] - o[0]), ty = (R)(X[1] - o[1]), tz = (R)(X[2] - o[2]);
  const V4* dr = dens + (int64_t)r * nt;
  const R kr = (R)k;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t e0 = 0; e0 < nt; e0 += EV_THREADS) {
    const int ne = (int)min((int64_t)EV_THREADS, nt - e0);
    __syncthreads();
    if (threadIdx.x < ne) {
      const int64_t j = e0 + threadIdx.x;
      for (int q = 0; q < 3; ++q) {
        V4 v;
        v.x = (R)(qpt[9 * j + 3 * q] - o[0]);
        v.y = (R)(qpt[9 * j + 3 * q + 1] - o[1]);
        v.z = (R)(qpt[9 * j + 3 * q + 2] - o[2]);
        v.w = (R)nrm[3 * j + q];
        s_q[threadIdx.x][q] = v;
      }
      const double h4 = 4.0 * hmax[j];
      V4 c;
      c.x = (R)(cent[3 * j] - o[0]);
      c.y = (R)(cent[3 * j + 1] - o[1]);
      c.z = (R)(cent[3 * j + 2] - o[2]);
      c.w = (R)(h4 * h4);
      s_c[threadIdx.x] = c;
      s_d[threadIdx.x] = dr[j];
    }
    __syncthreads();
    R g[6] = {0, 0, 0, 0, 0, 0};
    for (int e = 0; e < ne; ++e) {
      const V4 c = s_c[e];
      const R cx = c.x - tx, cy = c.y - ty, cz = c.z - tz;
      const V4 dd = s_d[e];
      if (cx * cx + cy * cy + cz * cz < c.w) {
        grad_near<R>(X, (int)(e0 + e), k, cent, qpt, nrm, area, hmax, dd, g);
        continue;
      }
      const V4 q0 = s_q[e][0], q1 = s_q[e][1], q2 = s_q[e][2];
      const R nx = q0.w, ny = q1.w, nz = q2.w;
      grad_eval<R>(q0.x - tx, q0.y - ty, q0.z - tz, nx, ny, nz, kr, dd.x, dd.y, dd.z, dd.w, g);
      grad_eval<R>(q1.x - tx, q1.y - ty, q1.z - tz, nx, ny, nz, kr, dd.x, dd.y, dd.z, dd.w, g);
      grad_eval<R>(q2.x - tx, q2.y - ty, q2.z - tz, nx, ny, nz, kr, dd.x, dd.y, dd.z, dd.w, g);
    }
    for (int c = 0; c < 6; ++c) acc[c] += (double)g[c];
  }
  if (live)
    for (int c = 0; c < 6; ++c) out[2 * (((int64_t)r * np + p) * nc + c0) + c] = (Rout)acc[c];
}

// ------------------------------------------- near leaves at field points --
// One warp per field point that has near leaves (the far pass's flag,
// compacted into near_list): the lanes walk the tree together and split the
// elements of every near leaf, each with the rule its distance calls for as
// in k_eval_points; the lanes' sums are reduced and added to the point's FP64
// far sums.  The stored P2P coordinates are relative to the element's leaf
// centre, so one FP64 difference per leaf (centre - x) places them relative
// to x; the target array's .w holds (4 h_j)^2 for the refined-rule test.
// The warps stride over the list, whose length is read on the device.
template <typename R, int MODE, int NR>
__global__ void __launch_bounds__(128) k_evf_near(int r0, int64_t nt, WalkTree wt, double k, int64_t np,
                                                  const double* __restrict__ pts, const int* __restrict__ tcs,
                                                  const int* __restrict__ near_list, const int* __restrict__ n_near,
                                                  const typename V4of<R>::T* __restrict__ tgt,
                                                  const typename V4of<R>::T* __restrict__ src,
                                                  const typename V4of<R>::T* __restrict__ dens,
                                                  const double* __restrict__ cent, const double* __restrict__ qpt,
                                                  const double* __restrict__ nrm, const double* __restrict__ area,
                                                  const double* __restrict__ hmax, const double* __restrict__ wgt,
                                                  int refine, double* __restrict__ acc) {
  typedef typename V4of<R>::T V4;
  constexpr bool VAL = MODE != 1, GRAD = MODE != 0;
  constexpr int NC = MODE == 0 ? 1 : (MODE == 1 ? 3 : 4);
  const int lane = threadIdx.x & 31;
  const int64_t nn = *n_near;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const R kr = (R)k;
  for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < nn; w += nw) {
    const int64_t i = near_list[w];
    const double X[3] = {pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]};
    const int t[3] = {tcs[3 * i], tcs[3 * i + 1], tcs[3 * i + 2]};
    R are[NR], aim[NR], g[NR][6];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      are[q] = aim[q] = 0;
#pragma unroll
      for (int c = 0; c < 6; ++c) g[q][c] = 0;
    }
    tree_walk(wt, t, [&](int kind, int l, int b) {
      if (kind != 1) return;
      const double* c = wt.lv[l].centre + 3 * b;
      const R sx = (R)(c[0] - X[0]), sy = (R)(c[1] - X[1]), sz = (R)(c[2] - X[2]);
      const int e1 = wt.lv[l].end[b];
      for (int j = wt.lv[l].start[b] + lane; j < e1; j += 32) {
        const V4 tc = tgt[j];
        const R cx = tc.x + sx, cy = tc.y + sy, cz = tc.z + sz;
        if (refine && cx * cx + cy * cy + cz * cz < tc.w) {
#pragma unroll
          for (int q = 0; q < NR; ++q) {
            const V4 dd = dens[(int64_t)(r0 + q) * nt + j];
            if (VAL) eval_near<R>(X, j, k, cent, qpt, nrm, area, hmax, wgt, dd, are[q], aim[q]);
            if (GRAD) grad_near<R>(X, j, k, cent, qpt, nrm, area, hmax, dd, g[q]);
          }
          continue;
        }
        const V4 q0 = src[3 * (int64_t)j], q1 = src[3 * (int64_t)j + 1], q2 = src[3 * (int64_t)j + 2];
        const R nx = q0.w, ny = q1.w, nz = q2.w;
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          const V4 dd = dens[(int64_t)(r0 + q) * nt + j];
          if (VAL) {
            p2p_eval(q0.x + sx, q0.y + sy, q0.z + sz, nx, ny, nz, kr, dd, are[q], aim[q]);
            p2p_eval(q1.x + sx, q1.y + sy, q1.z + sz, nx, ny, nz, kr, dd, are[q], aim[q]);
            p2p_eval(q2.x + sx, q2.y + sy, q2.z + sz, nx, ny, nz, kr, dd, are[q], aim[q]);
          }
          if (GRAD) {
            grad_eval<R>(q0.x + sx, q0.y + sy, q0.z + sz, nx, ny, nz, kr, dd.x, dd.y, dd.z, dd.w, g[q]);
            grad_eval<R>(q1.x + sx, q1.y + sy, q1.z + sz, nx, ny, nz, kr, dd.x, dd.y, dd.z, dd.w, g[q]);
            grad_eval<R>(q2.x + sx, q2.y + sy, q2.z + sz, nx, ny, nz, kr, dd.x, dd.y, dd.z, dd.w, g[q]);
          }
        }
      }
    });
    // the lanes' partial sums, reduced in the operator's precision
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      for (int o = 16; o > 0; o >>= 1) {
        if (VAL) {
          are[q] += __shfl_xor_sync(0xffffffffu, are[q], o);
          aim[q] += __shfl_xor_sync(0xffffffffu, aim[q], o);
        }
        if (GRAD)
#pragma unroll
          for (int c = 0; c < 6; ++c) g[q][c] += __shfl_xor_sync(0xffffffffu, g[q][c], o);
      }
      if (lane == 0) {
        double* a = acc + 2 * (((int64_t)(r0 + q) * np + i) * NC);
        int c0 = 0;
        if (VAL) {
          a[0] += (double)are[q];
          a[1] += (double)aim[q];
          c0 = 1;
        }
        if (GRAD)
#pragma unroll
          for (int c = 0; c < 6; ++c) a[2 * c0 + c] += (double)g[q][c];
      }
    }
  }
}

template <typename R, int MODE>
static int evf_near_impl(bem_handle* h, const WalkTree& wt, int nrhs, int64_t np, const double* pts, const int* tcs,
                         const int* near_list, const int* n_near, double* acc, int refine, cudaStream_t s) {
  typedef typename V4of<R>::T V4;
  const V4* tgt = (const V4*)(sizeof(R) == 4 ? (const void*)h->tgt32 : (const void*)h->tgt64);
  const V4* src = (const V4*)(sizeof(R) == 4 ? (const void*)h->src32 : (const void*)h->src64);
  // warps stride over the near list: enough blocks of 4 warps to fill the GPU
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((np + 3) / 4, (int64_t)h->nsm * 16));
  for (int r0 = 0; r0 < nrhs;) {
    const int rem = nrhs - r0;
#define EVF_NEAR(NRV)                                                                                          \
  k_evf_near<R, MODE, NRV><<<g, 128, 0, s>>>(r0, h->nt, wt, h->k, np, pts, tcs, near_list, n_near, tgt, src,     \
                                             (const V4*)h->dens, h->cent, h->qpt, h->nrm, h->area, h->hmax, h->wgt, \
                                             refine, acc);                                                     \
  r0 += NRV;
    if (rem >= 4) {
      EVF_NEAR(4)
    } else if (rem >= 2) {
      EVF_NEAR(2)
    } else {
      EVF_NEAR(1)
    }
#undef EVF_NEAR
    BEM_CUDA(cudaGetLastError());
  }
  return BEM_OK;
}

int bem_evf_near(bem_handle* h, const WalkTree& wt, int nrhs, int mode, int64_t np, const double* pts,
                 const int* tcs, const int* near_list, const int* n_near, double* acc, int refine,
                 cudaStream_t s) {
  const bool f64 = bem_is_fp64(h);
  if (mode == 0)
    return f64 ? evf_near_impl<double, 0>(h, wt, nrhs, np, pts, tcs, near_list, n_near, acc, refine, s)
               : evf_near_impl<float, 0>(h, wt, nrhs, np, pts, tcs, near_list, n_near, acc, refine, s);
  if (mode == 1)
    return f64 ? evf_near_impl<double, 1>(h, wt, nrhs, np, pts, tcs, near_list, n_near, acc, refine, s)
               : evf_near_impl<float, 1>(h, wt, nrhs, np, pts, tcs, near_list, n_near, acc, refine, s);
  return f64 ? evf_near_impl<double, 2>(h, wt, nrhs, np, pts, tcs, near_list, n_near, acc, refine, s)
             : evf_near_impl<float, 2>(h, wt, nrhs, np, pts, tcs, near_list, n_near, acc, refine, s);
}

// the FP64 sums of every point, back to the caller's order and dtype
template <typename Rout>
__global__ void k_evf_out(int64_t n, int64_t np, int nc, const int* __restrict__ perm, const double* __restrict__ acc,
                          Rout* __restrict__ out) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // over nrhs * np * nc complex values
  if (idx >= n) return;
  const int64_t c = idx % nc, i = (idx / nc) % np, r = idx / (nc * np);
  const int64_t o = ((r * np + perm[i]) * nc + c);
  out[2 * o] = (Rout)acc[2 * idx];
  out[2 * o + 1] = (Rout)acc[2 * idx + 1];
}

int bem_evf_out(int nrhs, int mode, int64_t np, const int* perm, const double* acc, int dtype, void* out,
                cudaStream_t s) {
  const int nc = mode == 0 ? 1 : (mode == 1 ? 3 : 4);
  const int64_t n = (int64_t)nrhs * np * nc;
  if (dtype == BEM_C128)
    k_evf_out<double><<<nblk(n, 256), 256, 0, s>>>(n, np, nc, perm, acc, (double*)out);
  else
    k_evf_out<float><<<nblk(n, 256), 256, 0, s>>>(n, np, nc, perm, acc, (float*)out);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

// the direct sum over all elements (mode 0: u, 1: grad u, 2: both)
template <typename R, typename Rout>
static int eval_direct(bem_handle* h, int nrhs, int mode, const double* points, int64_t npoints, void* out,
                       cudaStream_t s) {
  typedef typename V4of<R>::T V4;
  const dim3 grid((unsigned)((npoints + EV_THREADS - 1) / EV_THREADS), nrhs);
  const int nc = mode == 0 ? 1 : (mode == 1 ? 3 : 4);
  if (mode != 1) {
    k_eval_points<R, Rout><<<grid, EV_THREADS, 0, s>>>(h->nt, npoints, h->k, points, h->cent, h->qpt, h->nrm, h->area,
                                                       h->hmax, h->wgt, (const V4*)h->dens, nc, 0, (Rout*)out);
    BEM_CUDA(cudaGetLastError());
  }
  if (mode != 0) {
    k_eval_points_grad<R, Rout><<<grid, EV_THREADS, 0, s>>>(h->nt, npoints, h->k, points, h->cent, h->qpt, h->nrm,
                                                            h->area, h->hmax, (const V4*)h->dens, nc, mode == 2 ? 1 : 0,
                                                            (Rout*)out);
    BEM_CUDA(cudaGetLastError());
  }
  return BEM_OK;
}

extern "C" int bem_eval_points(bem_handle* h, int nrhs, int dtype, const void* x, const void* y,
                               const double* points, int64_t npoints, void* out, int flags, void* stream) {
  bem_set_error("");
  if (!h) return bem_fail(BEM_ERR_INVALID_ARG, "handle is NULL");
  if (nrhs < 1 || nrhs > h->nrhs_max) return bem_fail(BEM_ERR_INVALID_ARG, "nrhs out of [1, max_nrhs]");
  if (dtype != BEM_C64 && dtype != BEM_C128) return bem_fail(BEM_ERR_INVALID_ARG, "dtype must be BEM_C64 or BEM_C128");
  if (!x && !y) return bem_fail(BEM_ERR_INVALID_ARG, "x and y are both NULL");
  if (!points || !out || npoints < 1) return bem_fail(BEM_ERR_INVALID_ARG, "points and out required, npoints >= 1");
  if (flags & ~(BEM_EVAL_GRADIENT | BEM_EVAL_VALUE_GRADIENT | BEM_EVAL_DIRECT))
    return bem_fail(BEM_ERR_INVALID_ARG, "flags: BEM_EVAL_GRADIENT or BEM_EVAL_VALUE_GRADIENT, and BEM_EVAL_DIRECT");
  if ((flags & BEM_EVAL_GRADIENT) && (flags & BEM_EVAL_VALUE_GRADIENT))
    return bem_fail(BEM_ERR_INVALID_ARG, "BEM_EVAL_GRADIENT and BEM_EVAL_VALUE_GRADIENT exclude each other");
  if ((int64_t)(npoints + EV_THREADS - 1) / EV_THREADS > 0x7fffffffLL)
    return bem_fail(BEM_ERR_INVALID_ARG, "too many points for one call");
  const int mode = (flags & BEM_EVAL_VALUE_GRADIENT) ? 2 : ((flags & BEM_EVAL_GRADIENT) ? 1 : 0);
  cudaStream_t s = (cudaStream_t)stream;
  if (bem_is_fmm(h) && h->L >= 2 && !(flags & BEM_EVAL_DIRECT))
    return bem_eval_fmm(h, nrhs, dtype, x, y, points, npoints, out, mode, s);
  BEM_TRY(bem_prologue(h, nrhs, dtype, x, y, s));
  if (bem_is_fp64(h))
    return dtype == BEM_C128 ? eval_direct<double, double>(h, nrhs, mode, points, npoints, out, s)
                             : eval_direct<double, float>(h, nrhs, mode, points, npoints, out, s);
  return dtype == BEM_C128 ? eval_direct<float, double>(h, nrhs, mode, points, npoints, out, s)
                           : eval_direct<float, float>(h, nrhs, mode, points, npoints, out, s);
}

// ----------------------------------------------------------- point sources --
// b_i = sum_m a_m G(c_i - x_m), G = exp(ikr)/(4 pi r): the field of point
// sources at the collocation points, e.g. the adjoint right-hand side of
// Section 2.2 with weights a_m at the observation points.  One thread per
// element, FP64 (a handful of sources), written in the caller's order.
template <typename Rout>
__global__ void k_point_sources(int64_t nt, int nrhs, int nsrc, double k, const int* __restrict__ perm,
                                const double* __restrict__ cent, const double* __restrict__ pts,
                                const double* __restrict__ amps, Rout* __restrict__ out) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nt) return;
  const int64_t o = perm[s];
  const double c0 = cent[3 * s], c1 = cent[3 * s + 1], c2 = cent[3 * s + 2];
  for (int r = 0; r < nrhs; ++r) {
    double re = 0.0, im = 0.0;
    for (int m = 0; m < nsrc; ++m) {
      const double d0 = c0 - pts[3 * m], d1 = c1 - pts[3 * m + 1], d2 = c2 - pts[3 * m + 2];
      const double d = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      double sn, cs;
      sincos(k * d, &sn, &cs);
      const double g = 1.0 / (4.0 * BEM_PI * d);
      const double ar = amps[2 * ((int64_t)r * nsrc + m)], ai = amps[2 * ((int64_t)r * nsrc + m) + 1];
      re += g * (ar * cs - ai * sn);
      im += g * (ar * sn + ai * cs);
    }
    out[2 * ((int64_t)r * nt + o)] = (Rout)re;
    out[2 * ((int64_t)r * nt + o) + 1] = (Rout)im;
  }
}

extern "C" int bem_point_sources(bem_handle* h, int nrhs, int dtype, int nsrc, const double* points,
                                 const double* amps, void* out, void* stream) {
  bem_set_error("");
  if (!h) return bem_fail(BEM_ERR_INVALID_ARG, "handle is NULL");
  if (nrhs < 1 || nsrc < 1 || !points || !amps || !out)
    return bem_fail(BEM_ERR_INVALID_ARG, "nrhs, nsrc >= 1 and points, amps, out required");
  if (dtype != BEM_C64 && dtype != BEM_C128) return bem_fail(BEM_ERR_INVALID_ARG, "dtype must be BEM_C64 or BEM_C128");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nt = h->nt;
  const unsigned g = (unsigned)((nt + 255) / 256);
  if (dtype == BEM_C128)
    k_point_sources<double><<<g, 256, 0, s>>>(nt, nrhs, nsrc, h->k, h->perm, h->cent, points, amps, (double*)out);
  else
    k_point_sources<float><<<g, 256, 0, s>>>(nt, nrhs, nsrc, h->k, h->perm, h->cent, points, amps, (float*)out);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

// ---------------------------------------------- fields at arbitrary points --
// phi(x) = sum_m a_m G(x - x_m) at points x, with grad phi = sum_m a_m F(r) (x - x_m)
// (F = exp(ikr)(ikr - 1)/(4 pi r^3), r = |x - x_m|); FP64, one thread per point.
// out [nrhs][npts] or, with the gradient, [nrhs][npts][4]: (phi, d/dx, d/dy, d/dz).
__global__ void k_point_source_field(int nrhs, int nsrc, int64_t npts, double k, int grad,
                                     const double* __restrict__ src, const double* __restrict__ amps,
                                     const double* __restrict__ pts, double* __restrict__ out) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= npts) return;
  const double x0 = pts[3 * p], x1 = pts[3 * p + 1], x2 = pts[3 * p + 2];
  for (int r = 0; r < nrhs; ++r) {
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int m = 0; m < nsrc; ++m) {
      const double d0 = x0 - src[3 * m], d1 = x1 - src[3 * m + 1], d2 = x2 - src[3 * m + 2];
      const double rr = sqrt(d0 * d0 + d1 * d1 + d2 * d2), kr = k * rr;
      double sn, cs;
      sincos(kr, &sn, &cs);
      const double ar = amps[2 * ((int64_t)r * nsrc + m)], ai = amps[2 * ((int64_t)r * nsrc + m) + 1];
      const double g = 1.0 / (4.0 * BEM_PI * rr);
      const double er = ar * cs - ai * sn, ei = ar * sn + ai * cs;  // a exp(ikr)
      v[0] += g * er;
      v[1] += g * ei;
      // a F = a exp(ikr)(ikr - 1) / (4 pi r^3)
      const double f = g / (rr * rr);
      const double fr = f * (-er - kr * ei), fi = f * (kr * er - ei);
      v[2] += fr * d0;
      v[3] += fi * d0;
      v[4] += fr * d1;
      v[5] += fi * d1;
      v[6] += fr * d2;
      v[7] += fi * d2;
    }
    const int w = grad ? 4 : 1;
    for (int c = 0; c < 2 * w; ++c) out[2 * w * ((int64_t)r * npts + p) + c] = v[c];
  }
}

// T(x) = Re[c1 grad p . grad pa - c2 p pa] from the state and adjoint fields
// (complex128; field and gradient packed as [npts][4] complex)
__global__ void k_topological_derivative(int64_t npts, double c1, double c2, const double* __restrict__ st,
                                         const double* __restrict__ ad, double* __restrict__ T) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= npts) return;
  const double* a = st + 8 * p;
  const double* b = ad + 8 * p;
  double gg = 0.0;  // Re(grad p . grad pa)
  for (int c = 1; c < 4; ++c) gg += a[2 * c] * b[2 * c] - a[2 * c + 1] * b[2 * c + 1];
  const double pp = a[0] * b[0] - a[1] * b[1];
  T[p] = c1 * gg - c2 * pp;
}

extern "C" int bem_point_source_field(int nrhs, int nsrc, const double* src, const double* amps, int64_t npoints,
                                      const double* points, double k, int flags, double* out, void* stream) {
  bem_set_error("");
  if (nrhs < 1 || nsrc < 1 || npoints < 1 || !src || !amps || !points || !out || (flags & ~BEM_EVAL_GRADIENT))
    return bem_fail(BEM_ERR_INVALID_ARG, "nrhs, nsrc, npoints >= 1; src, amps, points, out required; flags 0 or "
                                         "BEM_EVAL_GRADIENT");
  cudaStream_t s = (cudaStream_t)stream;
  k_point_source_field<<<(unsigned)((npoints + 255) / 256), 256, 0, s>>>(
      nrhs, nsrc, npoints, k, (flags & BEM_EVAL_GRADIENT) ? 1 : 0, src, amps, points, out);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

extern "C" int bem_topological_derivative(int64_t npoints, double c1, double c2, const double* state,
                                          const double* adjoint, double* T, void* stream) {
  bem_set_error("");
  if (npoints < 1 || !state || !adjoint || !T) return bem_fail(BEM_ERR_INVALID_ARG, "npoints >= 1 and buffers");
  cudaStream_t s = (cudaStream_t)stream;
  k_topological_derivative<<<(unsigned)((npoints + 255) / 256), 256, 0, s>>>(npoints, c1, c2, state, adjoint, T);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

// ------------------------------------------------------------- correction --
// z_i += sum_j C^S_ij sigma_j - C^D_ij tau_j  (values pre-divided by the weight).
// One warp per row, accumulated in the operator's precision (FP32 in the mixed
// mode: about 130 terms per row, each already a small correction) and added to
// the FP64 near-field sum.  NR right-hand sides r0 + NR blockIdx.y + [0, NR)
// share each loaded value pair.
#define CORR_U 2
template <typename V4, typename R, int NR>
__global__ void k_correction(int64_t nt, int r0, const int* __restrict__ ptr, const int* __restrict__ col,
                             const V4* __restrict__ val, const V4* __restrict__ dens, double* __restrict__ zn) {
  int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  int r = r0 + blockIdx.y * NR;
  if (i >= nt) return;
  const V4* dr = dens + (int64_t)r * nt;
  R are[NR], aim[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) are[j] = aim[j] = 0;
  // the value and column loads of CORR_U entries per lane go out before any of
  // their density gathers (a row holds about 130 entries: two or three rounds)
  const int e1 = ptr[i + 1];
  for (int eb = ptr[i] + lane; eb < e1; eb += 32 * CORR_U) {
    V4 c[CORR_U];
    int cj[CORR_U];
#pragma unroll
    for (int u = 0; u < CORR_U; ++u) {
      const int e = eb + 32 * u;
      if (e < e1) {
        c[u] = val[e];
        cj[u] = col[e];
      }
    }
#pragma unroll
    for (int u = 0; u < CORR_U; ++u) {
      if (eb + 32 * u >= e1) break;
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        V4 d = dr[(int64_t)j * nt + cj[u]];
        are[j] += c[u].x * d.x - c[u].y * d.y - c[u].z * d.z + c[u].w * d.w;
        aim[j] += c[u].x * d.y + c[u].y * d.x - c[u].z * d.w - c[u].w * d.z;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    for (int o = 16; o > 0; o >>= 1) {
      are[j] += __shfl_xor_sync(0xffffffffu, are[j], o);
      aim[j] += __shfl_xor_sync(0xffffffffu, aim[j], o);
    }
    if (lane == 0) {
      int64_t o = 2 * ((int64_t)(r + j) * nt + i);
      zn[o] += (double)are[j];
      zn[o + 1] += (double)aim[j];
    }
  }
}

// -------------------------------------------------------------------- P2M --
template <typename R>
__global__ void k_p2m(int nleaf, const int* __restrict__ leafbox, int64_t nt, int P, const int* __restrict__ bstart,
                      const int* __restrict__ bend, const int64_t* __restrict__ row_off, const R* __restrict__ rows_ab,
                      const typename V4of<R>::T* __restrict__ dens, int64_t exp_base, int64_t exp_stride,
                      R* __restrict__ M) {
  typedef typename V4of<R>::T V4;
  int b = leafbox[blockIdx.x], r = blockIdx.y;
  const V4* dr = dens + (int64_t)r * nt;
  // the leaf's element rows follow each other, (P rounded up to even) coefficients apart
  const int64_t rb = row_off[bstart[b]], Pe = (P + 1) & ~1;
  for (int e = threadIdx.x; e < P; e += blockDim.x) {
    R are = 0, aim = 0;
    for (int j = bstart[b]; j < bend[b]; ++j) {
      const R* ab = rows_ab + 4 * (rb + (j - bstart[b]) * Pe);
      R a_re = ab[2 * e], a_im = ab[2 * e + 1];
      R b_re = ab[2 * (P + e)], b_im = ab[2 * (P + e) + 1];
      V4 d = dr[j];
      are += a_re * d.x - a_im * d.y - b_re * d.z + b_im * d.w;
      aim += a_re * d.y + a_im * d.x - b_re * d.w - b_im * d.z;
    }
    R* out = M + 2 * ((int64_t)r * exp_stride + exp_base + (int64_t)b * P + e);
    out[0] = are;
    out[1] = aim;
  }
}

// FP32: one thread per coefficient pair (2t, 2t+1) with 16-byte loads of the
// element rows, elements in rounds of P2M_U so that their loads are in flight
// together; NR right-hand sides r0 + NR blockIdx.y + [0, NR) share each row.
// A row [a (P complex) | b (P complex)] starts on a 16-byte boundary; b does
// too when P is even, otherwise it is read as two float2.
template <int NR>
__global__ void k_p2m_v(int nleaf, const int* __restrict__ leafbox, int64_t nt, int r0, int P,
                        const int* __restrict__ bstart, const int* __restrict__ bend,
                        const int64_t* __restrict__ row_off, const float* __restrict__ rows_ab,
                        const float4* __restrict__ dens, int64_t exp_base, int64_t exp_stride,
                        float* __restrict__ M) {
  const int b = leafbox[blockIdx.x], r = r0 + blockIdx.y * NR;
  const int e0 = 2 * threadIdx.x;
  if (e0 >= P) return;
  const bool two = e0 + 1 < P, peven = (P & 1) == 0;
  const float4* dr = dens + (int64_t)r * nt;
  float2 acc0[NR], acc1[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) acc0[q] = acc1[q] = make_float2(0.f, 0.f);
  const int j0 = bstart[b], j1 = bend[b];
  // the leaf's element rows follow each other, (P rounded up to even) coefficients apart
  const float* rows0 = rows_ab + 4 * row_off[j0];
  const int64_t Pe4 = 4 * (int64_t)((P + 1) & ~1);
  constexpr int P2M_U = NR == 1 ? 8 : 4;  // elements per round
  for (int jb = j0; jb < j1; jb += P2M_U) {
    float4 A[P2M_U], B[P2M_U], D[P2M_U][NR];
#pragma unroll
    for (int u = 0; u < P2M_U; ++u) {
      const int j = jb + u;
      if (j >= j1) {
        A[u] = B[u] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < NR; ++q) D[u][q] = A[u];
        continue;
      }
      const float* ab = rows0 + (int64_t)(j - j0) * Pe4;
      const float* bb = ab + 2 * P;
      if (two) {
        A[u] = *(const float4*)(ab + 2 * e0);
      } else {
        const float2 a2 = *(const float2*)(ab + 2 * e0);
        A[u] = make_float4(a2.x, a2.y, 0.f, 0.f);
      }
      if (peven) {
        B[u] = *(const float4*)(bb + 2 * e0);
      } else {
        const float2 b0 = *(const float2*)(bb + 2 * e0);
        const float2 b1 = two ? *(const float2*)(bb + 2 * e0 + 2) : make_float2(0.f, 0.f);
        B[u] = make_float4(b0.x, b0.y, b1.x, b1.y);
      }
#pragma unroll
      for (int q = 0; q < NR; ++q) D[u][q] = dr[(int64_t)q * nt + j];
    }
#pragma unroll
    for (int u = 0; u < P2M_U; ++u) {
      const float4 a = A[u], bq = B[u];
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        const float4 d = D[u][q];
        acc0[q].x += a.x * d.x - a.y * d.y - bq.x * d.z + bq.y * d.w;
        acc0[q].y += a.x * d.y + a.y * d.x - bq.x * d.w - bq.y * d.z;
        acc1[q].x += a.z * d.x - a.w * d.y - bq.z * d.z + bq.w * d.w;
        acc1[q].y += a.z * d.y + a.w * d.x - bq.z * d.w - bq.w * d.z;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    float* out = M + 2 * ((int64_t)(r + q) * exp_stride + exp_base + (int64_t)b * P + e0);
    out[0] = acc0[q].x;
    out[1] = acc0[q].y;
    if (two) {
      out[2] = acc1[q].x;
      out[3] = acc1[q].y;
    }
  }
}

// -------------------------------------------------------------------- L2P --
// One warp per target; NR right-hand sides r0 + NR blockIdx.y + [0, NR)
// share each loaded row.
template <typename R, int NR>
__device__ __forceinline__ void l2p_body(int64_t nt, int r0, const LevTab& lt, const int* __restrict__ leaf_of,
                                         const unsigned char* __restrict__ leaf_lev,
                                         const int64_t* __restrict__ row_off, const R* __restrict__ rows_r,
                                         const R* __restrict__ Lexp, int64_t exp_stride,
                                         double* __restrict__ zfar) {
  int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  int r = r0 + blockIdx.y * NR;
  if (i >= nt) return;
  int b = leaf_of[i];
  const int lvl = leaf_lev[i];
  const int P = lt.P[lvl];  // 0 for a leaf above level 2: no local expansion
  const R* row = rows_r + 2 * row_off[i];
  const R* Lb = Lexp + 2 * ((int64_t)r * exp_stride + lt.base[lvl] + (int64_t)b * P);
  const int64_t ls = 2 * exp_stride;  // between right-hand sides
  R are[NR], aim[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) are[q] = aim[q] = 0;
  if (sizeof(R) == 4 && (P & 1) == 0) {
    // P even: the row starts on a 16-byte boundary, two coefficients per load
    for (int e2 = lane; 2 * e2 < P; e2 += 32) {
      const float4 x = *(const float4*)((const float*)row + 4 * e2);
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        const float* Lq = (const float*)Lb + q * ls;
        const float2 l0 = *(const float2*)(Lq + 4 * e2);
        const float2 l1 = *(const float2*)(Lq + 4 * e2 + 2);
        are[q] += x.x * l0.x - x.y * l0.y + x.z * l1.x - x.w * l1.y;
        aim[q] += x.x * l0.y + x.y * l0.x + x.z * l1.y + x.w * l1.x;
      }
    }
  } else {
    for (int e = lane; e < P; e += 32) {
      R x = row[2 * e], y = row[2 * e + 1];
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        R lr = Lb[q * ls + 2 * e], li = Lb[q * ls + 2 * e + 1];
        are[q] += x * lr - y * li;
        aim[q] += x * li + y * lr;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    for (int o = 16; o > 0; o >>= 1) {
      are[q] += __shfl_xor_sync(0xffffffffu, are[q], o);
      aim[q] += __shfl_xor_sync(0xffffffffu, aim[q], o);
    }
    if (lane == 0) {
      int64_t o = 2 * ((int64_t)(r + q) * nt + i);
      zfar[o] = (double)are[q];
      zfar[o + 1] = (double)aim[q];
    }
  }
}

template <typename R, int NR>
__global__ void k_l2p(int64_t nt, int r0, LevTab lt, const int* __restrict__ leaf_of,
                      const unsigned char* __restrict__ leaf_lev, const int64_t* __restrict__ row_off,
                      const R* __restrict__ rows_r, const R* __restrict__ Lexp, int64_t exp_stride,
                      double* __restrict__ zfar) {
  l2p_body<R, NR>(nt, r0, lt, leaf_of, leaf_lev, row_off, rows_r, Lexp, exp_stride, zfar);
}
// FP32 with one right-hand side: eight blocks per SM, since the kernel is
// latency-bound on its row loads
__global__ void __launch_bounds__(256, 8) k_l2p_f1(int64_t nt, int r0, LevTab lt, const int* __restrict__ leaf_of,
                                                   const unsigned char* __restrict__ leaf_lev,
                                                   const int64_t* __restrict__ row_off,
                                                   const float* __restrict__ rows_r, const float* __restrict__ Lexp,
                                                   int64_t exp_stride, double* __restrict__ zfar) {
  l2p_body<float, 1>(nt, r0, lt, leaf_of, leaf_lev, row_off, rows_r, Lexp, exp_stride, zfar);
}

// ------------------------------------------------ grouped translation GEMM --
// For every job (group g, pairs [p0, p0+np), rows [row0, row0+BM)):
//   dst[dst_off[c] + Q_c(row)] += s_c(row) sum_k T_g[row][k] s_c(k) src[src_off[c] + Q_c(k)]
// where (Q_c, s_c) is the signed permutation of the pair's reflection flags:
// an x or y flip maps m -> -m (both flips cancel), an x flip contributes
// (-1)^m and a z flip (-1)^(n+m).  BM x BN complex output tile per CTA,
// 256 threads with TM x TN complex micro-tiles, K in chunks of 16 with the
// next chunk prefetched into registers while the current one is consumed.
template <typename R, int BM, int BN, int TM, int TN>
__global__ void __launch_bounds__(256) k_grouped_gemm(const int4* __restrict__ jobs, const int* __restrict__ grows,
                                                     const int* __restrict__ gcols, const int64_t* __restrict__ gmat,
                                                     const R* __restrict__ mats, const int* __restrict__ src_off,
                                                     const int* __restrict__ dst_off,
                                                     const unsigned char* __restrict__ pflags,
                                                     const R* __restrict__ src, R* __restrict__ dst,
                                                     int64_t exp_stride) {
  constexpr int BK = 16;
  constexpr int NTX = BN / TN;
  constexpr int AE = BM * BK / 256;  // A elements per thread per chunk
  constexpr int BE = BN * BK / 256;  // B elements per thread per chunk
  static_assert((BM / TM) * (BN / TN) == 256, "256 threads");
  __shared__ __align__(16) cpx<R> As[BK][BM + 2];
  __shared__ __align__(16) cpx<R> Bs[BK][BN + 2];
  __shared__ int s_src[BN], s_dst[BN], s_flg[BN];
  constexpr int KS = 128;  // K slice of one job
  int4 job = jobs[blockIdx.x];
  int r = blockIdx.y;
  int g = job.x, p0 = job.y, np = job.z & 255, row0 = job.w;
  int kbeg = (job.z >> 8) * KS;
  int rows = grows[g], cols = gcols[g];
  int kend = min(cols, kbeg + KS);
  const cpx<R>* T = (const cpx<R>*)(mats) + gmat[g];
  const cpx<R>* S = (const cpx<R>*)(src) + (int64_t)r * exp_stride;
  cpx<R>* D = (cpx<R>*)(dst) + (int64_t)r * exp_stride;
  int tid = threadIdx.x;
  for (int c = tid; c < BN; c += 256) {
    bool ok = c < np;
    s_src[c] = ok ? src_off[p0 + c] : -1;
    s_dst[c] = ok ? dst_off[p0 + c] : -1;
    s_flg[c] = ok ? (int)pflags[p0 + c] : 0;
  }
  int ty = tid / NTX, tx = tid % NTX;
  cpx<R> acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = cmk((R)0, (R)0);
  __syncthreads();
  cpx<R> ra[AE], rb[BE];
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < AE; ++q) {
      int e = tid + 256 * q;
      int row = row0 + e / BK, kk = k0 + e % BK;
      ra[q] = (row < rows && kk < kend) ? T[(int64_t)row * cols + kk] : cmk((R)0, (R)0);
    }
#pragma unroll
    for (int q = 0; q < BE; ++q) {
      int e = tid + 256 * q;
      int c = e / BK, kk = k0 + e % BK;
      cpx<R> v = cmk((R)0, (R)0);
      int so = s_src[c];
      if (so >= 0 && kk < kend) {
        bool neg;
        int ki = reflect_index(kk, s_flg[c], &neg);
        v = S[so + ki];
        if (neg) v = cmk(-v.re, -v.im);
      }
      rb[q] = v;
    }
  };
  load(kbeg);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int q = 0; q < AE; ++q) {
      int e = tid + 256 * q;
      As[e % BK][e / BK] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < BE; ++q) {
      int e = tid + 256 * q;
      Bs[e % BK][e / BK] = rb[q];
    }
    __syncthreads();
    if (k0 + BK < kend) load(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      cpx<R> a[TM], b[TN];
#pragma unroll
      for (int q = 0; q < TM; ++q) a[q] = As[kk][ty * TM + q];
#pragma unroll
      for (int q = 0; q < TN; ++q) b[q] = Bs[kk][tx * TN + q];
#pragma unroll
      for (int ii = 0; ii < TM; ++ii)
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) {
          acc[ii][jj].re += a[ii].re * b[jj].re - a[ii].im * b[jj].im;
          acc[ii][jj].im += a[ii].re * b[jj].im + a[ii].im * b[jj].re;
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int jj = 0; jj < TN; ++jj) {
    int c = tx * TN + jj;
    int dof = s_dst[c];
    if (dof < 0) continue;
    int fl = s_flg[c];
#pragma unroll
    for (int ii = 0; ii < TM; ++ii) {
      int row = row0 + ty * TM + ii;
      if (row < rows) {
        bool neg;
        int ri = reflect_index(row, fl, &neg);
        R* p = (R*)(D + dof + ri);
        atomicAdd(p, neg ? -acc[ii][jj].re : acc[ii][jj].re);
        atomicAdd(p + 1, neg ? -acc[ii][jj].im : acc[ii][jj].im);
      }
    }
  }
}

// ----------------------------------------------------------------- driver --
template <typename R>
static int run_grouped(bem_handle* h, GroupedOp& op, const void* src, void* dst, int nrhs, cudaStream_t s,
                       int* launches) {
  if (sizeof(R) == 4) return bem_run_grouped_tc(h, op, src, dst, nrhs, s, launches);  // tensor cores
  if (op.njobsA > 0) {
    dim3 grid(op.njobsA, nrhs);
    k_grouped_gemm<R, 64, 64, 4, 4><<<grid, 256, 0, s>>>(op.d_jobsA, op.d_group_rows, op.d_group_cols,
                                                         op.d_group_mat, (const R*)op.mats_base, op.d_src_off,
                                                         op.d_dst_off, op.d_flags, (const R*)src, (R*)dst,
                                                         h->exp_total);
    BEM_CUDA(cudaGetLastError());
    ++*launches;
  }
  if (op.njobsB > 0) {
    dim3 grid(op.njobsB, nrhs);
    k_grouped_gemm<R, 128, 16, 4, 2><<<grid, 256, 0, s>>>(op.d_jobsB, op.d_group_rows, op.d_group_cols,
                                                          op.d_group_mat, (const R*)op.mats_base, op.d_src_off,
                                                          op.d_dst_off, op.d_flags, (const R*)src, (R*)dst,
                                                          h->exp_total);
    BEM_CUDA(cudaGetLastError());
    ++*launches;
  }
  return BEM_OK;
}

// Calls f(NR, r0, nchunk) for the right-hand sides [0, nrhs): chunks of
// P2P_NR_MAX, then one chunk of the remainder.  Returns the launch count.
template <typename F>
static int by_rhs_chunks(int nrhs, F&& f) {
  static_assert(P2P_NR_MAX == 4, "remainder cases below assume chunks of 4");
  const int full = nrhs / 4, rem = nrhs - 4 * full;
  if (full) f(std::integral_constant<int, 4>(), 0, full);
  if (rem == 1) f(std::integral_constant<int, 1>(), 4 * full, 1);
  if (rem == 2) f(std::integral_constant<int, 2>(), 4 * full, 1);
  if (rem == 3) f(std::integral_constant<int, 3>(), 4 * full, 1);
  return (full > 0) + (rem > 0);
}

// P2M of every leaf level: h->dens into h->Mexp (which the caller zeroed)
template <typename R>
static int p2m_impl(bem_handle* h, int nrhs, cudaStream_t s, int* launches) {
  const int64_t nt = h->nt;
  const int L = h->L;
  const typename V4of<R>::T* dens = (const typename V4of<R>::T*)h->dens;
  int nl = 0;
  for (int l = 2; l <= L; ++l) {
    LevelInfo& lf = h->lev[l];
    if (lf.nleaf == 0) continue;
    if constexpr (sizeof(R) == 4) {
      nl += by_rhs_chunks(nrhs, [&](auto nr, int r0, int nchunk) {
        k_p2m_v<decltype(nr)::value><<<dim3(lf.nleaf, nchunk), ((lf.P + 1) / 2 + 31) / 32 * 32, 0, s>>>(
            lf.nleaf, lf.leafbox, nt, r0, lf.P, lf.start, lf.end, h->row_off, (const float*)h->p2m_rows,
            (const float4*)dens, lf.exp_base, h->exp_total, (float*)h->Mexp);
      });
    } else {
      nl += 1;
      k_p2m<R><<<dim3(lf.nleaf, nrhs), 128, 0, s>>>(lf.nleaf, lf.leafbox, nt, lf.P, lf.start, lf.end, h->row_off,
                                                    (const R*)h->p2m_rows, dens, lf.exp_base, h->exp_total,
                                                    (R*)h->Mexp);
    }
    BEM_CUDA(cudaGetLastError());
  }
  *launches += nl;
  return BEM_OK;
}

template <typename R>
static int apply_sorted_impl(bem_handle* h, int nrhs, cudaStream_t s) {
  typedef typename V4of<R>::T V4;
  int64_t nt = h->nt;
  const V4* dens = (const V4*)h->dens;
  const V4* tgt = (const V4*)(sizeof(R) == 4 ? (const void*)h->tgt32 : (const void*)h->tgt64);
  const V4* src = (const V4*)(sizeof(R) == 4 ? (const void*)h->src32 : (const void*)h->src64);
  bool fmm = bem_is_fmm(h);
  int L = h->L;
  // With p2p_ctas > 0 (FP32 FMM) the far field is forked first and the near
  // field runs beside it from p2p_ctas resident CTAs per SM.
  const bool overlap = fmm && L >= 2 && sizeof(R) == 4 && h->p2p_ctas > 0;
  auto near = [&]() -> int {
    int pr = bem_prof_begin(h, s);
    int nl = 1;
    if (fmm) {
      const unsigned gx = nblk(h->n_p2p_units, P2P_WARPS);
      if constexpr (sizeof(R) == 4) {
        if (overlap) {
          BEM_CUDA(cudaMemsetAsync(h->p2p_ctr, 0, sizeof(int) * (h->nrhs_max + 2), s));
          const unsigned gq = std::min<unsigned>(gx, (unsigned)(h->p2p_ctas * h->nsm));
          int c0 = 0;
          nl = by_rhs_chunks(nrhs, [&](auto nr, int r0, int nchunk) {
            k_p2p_fmm32_q<decltype(nr)::value><<<dim3(gq, nchunk), 32 * P2P_WARPS, 0, s>>>(
                h->n_p2p_units, nt, r0, (float)h->k, h->p2p_ctr + c0, h->p2p_units, h->u_ptr, h->u_src,
                h->u_shift32, h->gl_start, h->gl_end, (const float4*)tgt, (const float4*)src, (const float4*)dens,
                h->zn);
            c0 += nchunk;
          });
        } else if (h->p2p_stage) {
          nl = by_rhs_chunks(nrhs, [&](auto nr, int r0, int nchunk) {
            constexpr int NRV = decltype(nr)::value;
            const size_t sm = (size_t)P2P_WARPS * 2 * P2P_CH * (4 + NRV) * sizeof(float4);
            k_p2p_fmm32_s<NRV><<<dim3(gx, nchunk), 32 * P2P_WARPS, sm, s>>>(
                h->n_p2p_units, nt, r0, (float)h->k, h->p2p_units, h->u_ptr, h->u_src, h->u_shift32, h->gl_start,
                h->gl_end, (const float4*)tgt, (const float4*)src, (const float4*)dens, h->zn);
          });
        } else {
          nl = by_rhs_chunks(nrhs, [&](auto nr, int r0, int nchunk) {
            k_p2p_fmm32<decltype(nr)::value><<<dim3(gx, nchunk), 32 * P2P_WARPS, 0, s>>>(
                h->n_p2p_units, nt, r0, (float)h->k, h->p2p_units, h->u_ptr, h->u_src, h->u_shift32, h->gl_start,
                h->gl_end, (const float4*)tgt, (const float4*)src, (const float4*)dens, h->zn);
          });
        }
      } else {
        k_p2p_fmm64<<<dim3(gx, nrhs), 32 * P2P_WARPS, 0, s>>>(h->n_p2p_units, nt, h->k, h->p2p_units, h->u_ptr,
                                                            h->u_src, h->u_shift64, h->gl_start, h->gl_end,
                                                            (const double4*)tgt, (const double4*)src,
                                                            (const double4*)dens, h->zn);
      }
    } else {
      dim3 grid(nblk(nt, P2P_THREADS), nrhs);
      k_p2p_direct<R><<<grid, P2P_THREADS, 0, s>>>(nt, (R)h->k, tgt, src, dens, h->zn);
    }
    BEM_CUDA(cudaGetLastError());
    bem_prof_end(h, pr, 1, nl, s);
    return BEM_OK;
  };
  int pr, nl;
  if (!overlap) BEM_TRY(near());
  if (!fmm || L < 2) {
    pr = bem_prof_begin(h, s);
    nl = by_rhs_chunks(nrhs, [&](auto nr, int r0, int nchunk) {
      k_correction<V4, R, decltype(nr)::value><<<dim3(nblk(nt * 32, 256), nchunk), 256, 0, s>>>(
          nt, r0, h->corr_ptr, h->corr_col, (const V4*)h->corr_val, dens, h->zn);
    });
    BEM_CUDA(cudaGetLastError());
    bem_prof_end(h, pr, 2, nl, s);
    BEM_CUDA(cudaMemsetAsync(h->zfar, 0, sizeof(double) * 2 * nt * nrhs, s));
    return BEM_OK;
  }
  auto far = [&](cudaStream_t s) -> int {
    int pr, nl;
    // far field
    size_t esz = 2 * sizeof(R);
    const LevTab lt = bem_levtab(h);
    pr = bem_prof_begin(h, s);
    BEM_CUDA(cudaMemsetAsync(h->Mexp, 0, esz * h->exp_total * nrhs, s));
    BEM_CUDA(cudaMemsetAsync(h->Lexp, 0, esz * h->exp_total * nrhs, s));
    nl = 0;
    BEM_TRY(p2m_impl<R>(h, nrhs, s, &nl));
    bem_prof_end(h, pr, 3, nl, s);
    nl = 0;
    pr = bem_prof_begin(h, s);
    for (int l = L - 1; l >= 2; --l) BEM_TRY(run_grouped<R>(h, h->m2m[l], h->Mexp, h->Mexp, nrhs, s, &nl));
    bem_prof_end(h, pr, 4, nl, s);
    nl = 0;
    pr = bem_prof_begin(h, s);
    for (int l = 2; l <= L; ++l) BEM_TRY(run_grouped<R>(h, h->m2l[l], h->Mexp, h->Lexp, nrhs, s, &nl));
    BEM_TRY(bem_run_p2l(h, nrhs, dens, h->Lexp, s, &nl));  // X-lists, before the local expansions go down
    bem_prof_end(h, pr, 5, nl, s);
    nl = 0;
    pr = bem_prof_begin(h, s);
    for (int l = 2; l < L; ++l) BEM_TRY(run_grouped<R>(h, h->l2l[l], h->Lexp, h->Lexp, nrhs, s, &nl));
    bem_prof_end(h, pr, 6, nl, s);
    pr = bem_prof_begin(h, s);
    nl = by_rhs_chunks(nrhs, [&](auto nr, int r0, int nchunk) {
      const dim3 grid(nblk(nt * 32, 256), nchunk);
      if constexpr (sizeof(R) == 4 && decltype(nr)::value == 1)
        k_l2p_f1<<<grid, 256, 0, s>>>(nt, r0, lt, h->leaf_of, h->leaf_lev, h->row_off, (const float*)h->l2p_rows,
                                      (const float*)h->Lexp, h->exp_total, h->zfar);
      else
        k_l2p<R, decltype(nr)::value><<<grid, 256, 0, s>>>(nt, r0, lt, h->leaf_of, h->leaf_lev, h->row_off,
                                                           (const R*)h->l2p_rows, (const R*)h->Lexp, h->exp_total,
                                                           h->zfar);
    });
    BEM_CUDA(cudaGetLastError());
    BEM_TRY(bem_run_m2p(h, nrhs, h->Mexp, h->zfar, s, &nl));  // W-lists, added to the far sums
    bem_prof_end(h, pr, 7, nl, s);
    return BEM_OK;
  };
  // After the P2P, the far field runs on the handle's high-priority second
  // stream beside the correction (40,960 short CTAs that would otherwise fill
  // the SMs ahead of the translation chain's small launches); both join back
  // into `s`.  The P2P itself stays alone: its long-lived CTAs fill the
  // registers of every SM, and a far field forked before it waited for them.
  BEM_CUDA(cudaEventRecord(h->ev_fork, s));
  BEM_CUDA(cudaStreamWaitEvent(h->s_far, h->ev_fork, 0));
  const int rc = far(h->s_far);
  if (overlap) {
    const int rn = near();
    if (rn != BEM_OK) {
      cudaEventRecord(h->ev_join, h->s_far);
      cudaStreamWaitEvent(s, h->ev_join, 0);
      return rn;
    }
  }
  pr = bem_prof_begin(h, s);
  nl = by_rhs_chunks(nrhs, [&](auto nr, int r0, int nchunk) {
    k_correction<V4, R, decltype(nr)::value><<<dim3(nblk(nt * 32, 256), nchunk), 256, 0, s>>>(
        nt, r0, h->corr_ptr, h->corr_col, (const V4*)h->corr_val, dens, h->zn);
  });
  BEM_CUDA(cudaGetLastError());
  bem_prof_end(h, pr, 2, nl, s);
  cudaError_t e = cudaEventRecord(h->ev_join, h->s_far);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_join, 0);
  BEM_TRY(rc);
  BEM_CUDA(e);
  return BEM_OK;
}

int bem_run_grouped(bem_handle* h, GroupedOp& op, const void* src, void* dst, int nrhs, cudaStream_t s,
                    int* launches) {
  if (bem_is_fp64(h)) return run_grouped<double>(h, op, src, dst, nrhs, s, launches);
  return run_grouped<float>(h, op, src, dst, nrhs, s, launches);
}

template <typename R>
static int upward_impl(bem_handle* h, int nrhs, cudaStream_t s) {
  BEM_CUDA(cudaMemsetAsync(h->Mexp, 0, 2 * sizeof(R) * h->exp_total * nrhs, s));
  int nl = 0;
  BEM_TRY(p2m_impl<R>(h, nrhs, s, &nl));
  for (int l = h->L - 1; l >= 2; --l) BEM_TRY(run_grouped<R>(h, h->m2m[l], h->Mexp, h->Mexp, nrhs, s, &nl));
  return BEM_OK;
}

int bem_run_upward(bem_handle* h, int nrhs, cudaStream_t s) {
  if (bem_is_fp64(h)) return upward_impl<double>(h, nrhs, s);
  return upward_impl<float>(h, nrhs, s);
}

int bem_apply_sorted(bem_handle* h, int nrhs, cudaStream_t s) {
  if (bem_is_fp64(h)) return apply_sorted_impl<double>(h, nrhs, s);
  return apply_sorted_impl<float>(h, nrhs, s);
}

int bem_prologue(bem_handle* h, int nrhs, int dtype, const void* x, const void* y, cudaStream_t s) {
  int64_t nt = h->nt;
  unsigned g = nblk(nt, 256);
  bool f64 = bem_is_fp64(h);
  if (dtype == BEM_C128) {
    if (f64)
      k_prologue<double, double4><<<g, 256, 0, s>>>(nt, nrhs, h->perm, h->wgt, (const double*)x, (const double*)y,
                                                    (double4*)h->dens);
    else
      k_prologue<double, float4><<<g, 256, 0, s>>>(nt, nrhs, h->perm, h->wgt, (const double*)x, (const double*)y,
                                                   (float4*)h->dens);
  } else {
    if (f64)
      k_prologue<float, double4><<<g, 256, 0, s>>>(nt, nrhs, h->perm, h->wgt, (const float*)x, (const float*)y,
                                                   (double4*)h->dens);
    else
      k_prologue<float, float4><<<g, 256, 0, s>>>(nt, nrhs, h->perm, h->wgt, (const float*)x, (const float*)y,
                                                  (float4*)h->dens);
  }
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

int bem_epilogue(bem_handle* h, int nrhs, int dtype, const void* x, void* z, int half, cudaStream_t s) {
  int64_t nt = h->nt;
  unsigned g = nblk(nt, 256);
  if (dtype == BEM_C128)
    k_epilogue<double, double><<<g, 256, 0, s>>>(nt, nrhs, h->perm, (const double*)x, half, h->zn, h->zfar,
                                                 (double*)z);
  else
    k_epilogue<float, float><<<g, 256, 0, s>>>(nt, nrhs, h->perm, (const float*)x, half, h->zn, h->zfar, (float*)z);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}
