// bem_grad_vertices.cu -- derivative of a real loss with respect to the vertex
// positions of the mesh (the shape gradient the topology optimisation of
// Section 2.5 needs, restricted here to the boundary operators of Section 2.3).
//
// For z = (1/2 I - D) x + S y and the upstream gradient g (PyTorch's complex
// convention), dL = sum_rhs sum_i Re(conj(g_i) dz_i).  The 1/2 I term does not
// move with the mesh, so per pair (i, j), with cy = sum_rhs conj(g_i) y_j and
// cx = sum_rhs conj(g_i) x_j, the loss holds l_ij = Re(cy S_ij - cx D_ij).
//
// One point y of weight w on Gamma_j seen from the collocation point x:
//   d = y - x, r = |d|, E = exp(ikr)/(4 pi)
//   G = E/r                         (the single-layer kernel)
//   F = E (ikr - 1)/r^3             grad_y G = F d,  dG/dn_y = F (d.n)
//   H = E (3 - 3ikr - k^2 r^2)/r^5  grad_y F = H d
//   grad_y (dG/dn_y) = H (d.n) d + F n;  grad_x = -grad_y for both kernels.
// The entry also moves through the weight (w = A/(3 4^L), A the area) and the
// unit normal n.  With e_a = V_{a+1} - V_{a+2} (cyclic vertex order) and
// P = I - n n^T:
//   dA/dV_a = (1/2) e_a x n,     d(u.n)/dV_a = e_a x (P u) / (2 A),
// and the point y = sum_a beta_a V_a moves with the vertices by beta_a.  The
// collocation point is the centroid, so it moves by 1/3 with each vertex of
// its own triangle.
//
// Pieces, all on the stream:
//   regular rule R_0 over every pair: one target-major pass gives the centroid
//     gradients, one source-major pass the point / area / normal gradients.
//     FP64 in the FP64 modes; otherwise FP32 with block-relative coordinates
//     split into high and low FP32 parts (separations keep FP32 relative
//     accuracy at any distance) and FP64 accumulation after every 32 sources.
//   corrections: for every pair of the correction matrix, the derivative of
//     the refined rule R_L, or of the exact self term, minus that of R_0; FP64
//     in the FP64 modes and for the self terms, FP32 relative to the
//     collocation point for the other pairs of the mixed modes.  The exact self term S_ii (D_ii = 0 for every vertex
//     position) differentiates in closed radial form: with lambda_a the
//     barycentric coordinates and polar coordinates (rho, u) about the centroid,
//       dS_ii/dV_a = (dA/dV_a) S_ii / A
//                  + (1/4 pi) int u (u . grad lambda_a) K(R(phi)) dphi,
//       K(R) = int_0^R exp(ik rho)(ik rho - 1) d rho = R exp(ikR) - 2 (exp(ikR) - 1)/(ik),
//     integrated per edge with the substitution tan(phi) = sinh(t) and 32-point
//     Gauss-Legendre on panels of length <= 4 in t.
//   finish: per element, everything mapped onto its three vertices and added
//     into the caller's vertex order.
#include <type_traits>

#include "bem_common.cuh"
#include "bem_tree_walk.cuh"

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// sin/cos in the precision of the pair evaluation
__device__ __forceinline__ void sc(float a, float* s, float* c) { sincosf(a, s, c); }
__device__ __forceinline__ void sc(double a, double* s, double* c) { sincos(a, s, c); }

// G, F, H of one point at separation d (|d| > 0)
template <typename R>
__device__ __forceinline__ void ghfr(R d0, R d1, R d2, R k, cpx<R>& G, cpx<R>& F, cpx<R>& H, R& r) {
  R r2 = d0 * d0 + d1 * d1 + d2 * d2;
  r = sqrt(r2);
  R ir = R(1) / r;
  R ir2 = ir * ir;
  R kr = k * r;
  R sn, cs;
  sc(kr, &sn, &cs);
  const R c4 = R(1.0 / (4.0 * BEM_PI));
  cpx<R> E = cmk(cs * c4, sn * c4);
  G = ir * E;
  // F = E (ikr - 1) / r^3
  F = (ir * ir2) * (E * cmk(R(-1), kr));
  // H = E (3 - k^2 r^2 - 3ikr) / r^5
  H = (ir2 * ir2 * ir) * (E * cmk(R(3) - kr * kr, R(-3) * kr));
}
template <typename R>
__device__ __forceinline__ void ghf(R d0, R d1, R d2, R k, cpx<R>& G, cpx<R>& F, cpx<R>& H) {
  R r;
  ghfr(d0, d1, d2, k, G, F, H, r);
}

// ------------------------------------------------------ regular rule R_0 --
// In the FP32 passes every coordinate relative to the block's reference point
// is held as a high FP32 part and the FP32 rounding of the rest, and a
// separation is formed as (q_hi - x_hi) + (q_lo - x_lo): the difference of the
// high parts is exact up to one rounding of the separation itself, so a pair a
// fraction of an edge apart keeps FP32 relative accuracy although both points
// lie many edges from the reference.  The FP32 sums are moved to FP64 after
// every 32 sources.

// Target-major pass: for every collocation point x_i,
//   gx_i += Re( conj(g_i) sum_j sum_q w_j [ -F d y_j + (H (d.n) d + F n) x_j ] ),
// the gradient of l_i = sum_j l_ij with respect to x_i (w_j = A_j/3).  One
// thread per target, sources streamed through shared memory; coordinates are
// taken relative to the block's first centroid before rounding to R.  Block z
// takes the sources [z chunk, (z + 1) chunk) and adds its partial sums.  With
// GX false only the regular part of dL/dk is summed (the tree gives gx, or
// only dL/dk is asked for), with the same arithmetic.
template <typename R, bool GX>
__global__ void __launch_bounds__(128) k_gv_target(int64_t nt, double k, const double* __restrict__ cent,
                                                   const double* __restrict__ qpt, const double* __restrict__ nrm,
                                                   const double* __restrict__ area, const double4* __restrict__ yx,
                                                   const double2* __restrict__ gs, int64_t chunk,
                                                   double* __restrict__ gx, double* __restrict__ dk) {
  constexpr bool F32 = sizeof(R) == 4;
  __shared__ R s_q[128][9];
  __shared__ float s_ql[F32 ? 128 : 1][9];  // FP32 only: low parts of s_q
  __shared__ R s_n[128][3];
  __shared__ cpx<R> s_y[128], s_x[128];
  const int r = blockIdx.y;
  const int64_t i0 = blockIdx.x * (int64_t)128;
  const int64_t i = i0 + threadIdx.x;
  double ref[3];
  for (int d = 0; d < 3; ++d) ref[d] = cent[3 * i0 + d];
  R x[3] = {R(0), R(0), R(0)};
  float xl[3] = {0.f, 0.f, 0.f};
  if (i < nt)
    for (int d = 0; d < 3; ++d) {
      const double v = cent[3 * i + d] - ref[d];
      x[d] = R(v);
      xl[d] = (float)(v - (double)x[d]);
    }
  const double4* u = yx + (int64_t)r * nt;
  const R kk = R(k);
  double acc[6] = {0, 0, 0, 0, 0, 0};
  double kacc[2] = {0, 0};  // sum of w [dS/dk y_j - dD/dk x_j] over the pairs of this target
  const int64_t ebeg = blockIdx.z * chunk, eend = min(nt, ebeg + chunk);
  for (int64_t e0 = ebeg; e0 < eend; e0 += 128) {
    const int ne = (int)min((int64_t)128, eend - e0);
    __syncthreads();
    if (threadIdx.x < ne) {
      const int64_t j = e0 + threadIdx.x;
      for (int m = 0; m < 9; ++m) {
        const double v = qpt[9 * j + m] - ref[m % 3];
        s_q[threadIdx.x][m] = R(v);
        if constexpr (F32) s_ql[threadIdx.x][m] = (float)(v - (double)s_q[threadIdx.x][m]);
      }
      for (int d = 0; d < 3; ++d) s_n[threadIdx.x][d] = R(nrm[3 * j + d]);
      const double w = area[j] / 3.0;
      const double4 v = u[j];
      s_y[threadIdx.x] = cmk(R(w * v.x), R(w * v.y));
      s_x[threadIdx.x] = cmk(R(w * v.z), R(w * v.w));
    }
    __syncthreads();
    if (i < nt) {
      for (int c0 = 0; c0 < ne; c0 += 32) {
        const int c1 = min(ne, c0 + 32);
        cpx<R> T0 = cmk(R(0), R(0)), T1 = T0, T2 = T0, KT = T0;
        for (int e = c0; e < c1; ++e) {
          const cpx<R> wy = s_y[e], wx = s_x[e];
          const R n0 = s_n[e][0], n1 = s_n[e][1], n2 = s_n[e][2];
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            R d0 = s_q[e][3 * q] - x[0], d1 = s_q[e][3 * q + 1] - x[1], d2 = s_q[e][3 * q + 2] - x[2];
            if constexpr (F32) {
              d0 += s_ql[e][3 * q] - xl[0];
              d1 += s_ql[e][3 * q + 1] - xl[1];
              d2 += s_ql[e][3 * q + 2] - xl[2];
            }
            const R dn = d0 * n0 + d1 * n1 + d2 * n2;
            cpx<R> G, F, H;
            R rr;
            ghfr(d0, d1, d2, kk, G, F, H, rr);
            // d/dk: G (i r w y + k (d.n) w x)
            KT = KT + G * (cmk(-rr * wy.im, rr * wy.re) + (kk * dn) * wx);
            if constexpr (GX) {
              const cpx<R> a = dn * (H * wx) - F * wy;
              const cpx<R> b = F * wx;
              T0 = T0 + d0 * a + n0 * b;
              T1 = T1 + d1 * a + n1 * b;
              T2 = T2 + d2 * a + n2 * b;
            }
          }
        }
        acc[0] += T0.re;
        acc[1] += T0.im;
        acc[2] += T1.re;
        acc[3] += T1.im;
        acc[4] += T2.re;
        acc[5] += T2.im;
        kacc[0] += KT.re;
        kacc[1] += KT.im;
      }
    }
  }
  double kpart = 0.0;
  if (i < nt) {
    const double2 g = gs[(int64_t)r * nt + i];
    if constexpr (GX)
      for (int d = 0; d < 3; ++d) atomicAdd(&gx[3 * i + d], g.x * acc[2 * d] + g.y * acc[2 * d + 1]);
    kpart = g.x * kacc[0] + g.y * kacc[1];  // Re(conj(g_i) K_i)
  }
  if (dk) {
    __shared__ double s_red[128];
    s_red[threadIdx.x] = kpart;
    __syncthreads();
    for (int st = 64; st > 0; st >>= 1) {
      if (threadIdx.x < st) s_red[threadIdx.x] += s_red[threadIdx.x + st];
      __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(dk, s_red[0]);
  }
}

// Source-major pass: one thread per quadrature point p = 3 j + q of the regular
// rule, the collocation points [z chunk, (z + 1) chunk) of block z streamed
// through shared memory (partial sums added).  With
// c_i = conj(g_i) it sums PS = sum c F d, QH = sum c H (d.n) d, Fs = sum c F,
// GS = sum c G, GD = sum c F (d.n) and leaves
//   gq[p] = Re( w (y_j PS - x_j (QH + Fs n)) )   (gradient w.r.t. the point)
//   ga[j] += Re( y_j GS - x_j GD ) / 3           (w.r.t. the area, w/A = 1/3)
//   gn[j] += -Re( w x_j PS )                     (w.r.t. the unit normal)
template <typename R>
__global__ void __launch_bounds__(128) k_gv_source(int64_t nt, double k, const double* __restrict__ cent,
                                                   const double* __restrict__ qpt, const double* __restrict__ nrm,
                                                   const double* __restrict__ area, const double4* __restrict__ yx,
                                                   const double2* __restrict__ gs, int64_t chunk,
                                                   double* __restrict__ gq, double* __restrict__ ga,
                                                   double* __restrict__ gn) {
  constexpr bool F32 = sizeof(R) == 4;
  __shared__ R s_x[128][3];
  __shared__ float s_xl[F32 ? 128 : 1][3];  // FP32 only: low parts of s_x
  __shared__ cpx<R> s_g[128];
  const int r = blockIdx.y;
  const int64_t p0 = blockIdx.x * (int64_t)128;
  const int64_t p = p0 + threadIdx.x;
  const bool act = p < 3 * nt;
  const int64_t j = act ? p / 3 : 0;
  const int q = (int)(p % 3);
  double ref[3];
  for (int d = 0; d < 3; ++d) ref[d] = cent[3 * (p0 / 3) + d];
  R y[3], n[3];
  float yl[3];
  for (int d = 0; d < 3; ++d) {
    const double v = qpt[9 * j + 3 * q + d] - ref[d];
    y[d] = R(v);
    yl[d] = (float)(v - (double)y[d]);
    n[d] = R(nrm[3 * j + d]);
  }
  const R kk = R(k);
  const double2* gr = gs + (int64_t)r * nt;
  double PS[6] = {0, 0, 0, 0, 0, 0}, QH[6] = {0, 0, 0, 0, 0, 0}, Fs[2] = {0, 0}, GS[2] = {0, 0}, GD[2] = {0, 0};
  const int64_t ebeg = blockIdx.z * chunk, eend = min(nt, ebeg + chunk);
  for (int64_t e0 = ebeg; e0 < eend; e0 += 128) {
    const int ne = (int)min((int64_t)128, eend - e0);
    __syncthreads();
    if (threadIdx.x < ne) {
      const int64_t i = e0 + threadIdx.x;
      for (int d = 0; d < 3; ++d) {
        const double v = cent[3 * i + d] - ref[d];
        s_x[threadIdx.x][d] = R(v);
        if constexpr (F32) s_xl[threadIdx.x][d] = (float)(v - (double)s_x[threadIdx.x][d]);
      }
      const double2 g = gr[i];
      s_g[threadIdx.x] = cmk(R(g.x), R(-g.y));
    }
    __syncthreads();
    if (act) {
      for (int c0 = 0; c0 < ne; c0 += 32) {
        const int c1 = min(ne, c0 + 32);
        cpx<R> ps0 = cmk(R(0), R(0)), ps1 = ps0, ps2 = ps0, qh0 = ps0, qh1 = ps0, qh2 = ps0, fs = ps0,
               gsum = ps0, gd = ps0;
        for (int e = c0; e < c1; ++e) {
          R d0 = y[0] - s_x[e][0], d1 = y[1] - s_x[e][1], d2 = y[2] - s_x[e][2];
          if constexpr (F32) {
            d0 += yl[0] - s_xl[e][0];
            d1 += yl[1] - s_xl[e][1];
            d2 += yl[2] - s_xl[e][2];
          }
          cpx<R> G, F, H;
          ghf(d0, d1, d2, kk, G, F, H);
          const R dn = d0 * n[0] + d1 * n[1] + d2 * n[2];
          const cpx<R> c = s_g[e];
          const cpx<R> cF = c * F;
          const cpx<R> cH = dn * (c * H);
          ps0 = ps0 + d0 * cF;
          ps1 = ps1 + d1 * cF;
          ps2 = ps2 + d2 * cF;
          qh0 = qh0 + d0 * cH;
          qh1 = qh1 + d1 * cH;
          qh2 = qh2 + d2 * cH;
          fs = fs + cF;
          gsum = gsum + c * G;
          gd = gd + dn * cF;
        }
        PS[0] += ps0.re; PS[1] += ps0.im; PS[2] += ps1.re; PS[3] += ps1.im; PS[4] += ps2.re; PS[5] += ps2.im;
        QH[0] += qh0.re; QH[1] += qh0.im; QH[2] += qh1.re; QH[3] += qh1.im; QH[4] += qh2.re; QH[5] += qh2.im;
        Fs[0] += fs.re; Fs[1] += fs.im;
        GS[0] += gsum.re; GS[1] += gsum.im;
        GD[0] += gd.re; GD[1] += gd.im;
      }
    }
  }
  if (!act) return;
  const double w = area[j] / 3.0;
  const double4 v = yx[(int64_t)r * nt + j];
  const zd yj = cmk(v.x, v.y), xj = cmk(v.z, v.w);
  const zd fsz = cmk(Fs[0], Fs[1]);
  for (int d = 0; d < 3; ++d) {
    const zd ps = cmk(PS[2 * d], PS[2 * d + 1]);
    const zd qh = cmk(QH[2 * d], QH[2 * d + 1]) + nrm[3 * j + d] * fsz;
    const zd t = yj * ps - xj * qh;
    atomicAdd(&gq[3 * p + d], w * t.re);
    atomicAdd(&gn[3 * j + d], -w * (xj * ps).re);
  }
  const zd ar = yj * cmk(GS[0], GS[1]) - xj * cmk(GD[0], GD[1]);
  atomicAdd(&ga[j], ar.re / 3.0);
}

// ------------------------------------------------------------ corrections --
template <typename R>
struct VTriT {
  R v[3][3], n[3], c[3], area, h;
};
typedef VTriT<double> VTri;

__device__ void vload(const double* __restrict__ qpt, const double* __restrict__ nrm, const double* __restrict__ cent,
                      const double* __restrict__ area, const double* __restrict__ hmax, int64_t j, VTri& t) {
  for (int d = 0; d < 3; ++d) {
    t.c[d] = cent[3 * j + d];
    t.n[d] = nrm[3 * j + d];
  }
  // the rule's point a is (2/3) V_a + (1/6)(V_b + V_c) = (V_a + 3 c)/2
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) t.v[a][d] = 2.0 * qpt[9 * j + 3 * a + d] - t.c[d];
  t.area = area[j];
  t.h = hmax[j];
}

template <typename R>
__device__ __forceinline__ void cross(const R* a, const R* b, R* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// adds dL/dA (scalar) and dL/dn (vector) of triangle t onto its vertices
template <typename R>
__device__ void map_area_normal(const VTriT<R>& t, R gA, const R* gN, R* g9) {
  R nn = gN[0] * t.n[0] + gN[1] * t.n[1] + gN[2] * t.n[2];
  R pg[3] = {gN[0] - nn * t.n[0], gN[1] - nn * t.n[1], gN[2] - nn * t.n[2]};
  for (int a = 0; a < 3; ++a) {
    const R* b = t.v[(a + 1) % 3];
    const R* c = t.v[(a + 2) % 3];
    R e[3] = {b[0] - c[0], b[1] - c[1], b[2] - c[2]};
    R ea[3], en[3];
    cross(e, t.n, ea);
    cross(e, pg, en);
    for (int d = 0; d < 3; ++d) g9[3 * a + d] += R(0.5) * gA * ea[d] + en[d] / (R(2) * t.area);
  }
}

// sign * d/d(geometry) of Re(cy S_ij - cx D_ij) under rule R_L on triangle t:
// the collocation point's gradient goes to tgt, the vertices' to g9.  With kd
// non-null the same points also add sign * (dS_ij/dk, dD_ij/dk) to kd[0],
// kd[1]: w i r G and -w k (d.n) G per point.
template <typename R>
__device__ void rule_grad(const R* x, const VTriT<R>& t, int L, R k, cpx<R> cy, cpx<R> cx, R sign, R* tgt, R* g9,
                          cpx<R>* kd = nullptr) {
  const int npieces = 1 << (2 * L);
  const R w = t.area / (R(3) * npieces);
  R gA = 0, gN[3] = {0, 0, 0};
  R g9l[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, tl[3] = {0, 0, 0};
  for (int piece = 0; piece < npieces; ++piece) {
    // barycentric coordinates (rows: the piece's corners, columns: V_0..V_2)
    R B[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    int code = piece;
    for (int lvl = 0; lvl < L; ++lvl) {
      const int child = code & 3;
      code >>= 2;
      R ab[3], bc[3], ca[3];
      for (int a = 0; a < 3; ++a) {
        ab[a] = R(0.5) * (B[0][a] + B[1][a]);
        bc[a] = R(0.5) * (B[1][a] + B[2][a]);
        ca[a] = R(0.5) * (B[2][a] + B[0][a]);
      }
      for (int a = 0; a < 3; ++a) {
        if (child == 0) {
          B[1][a] = ab[a];
          B[2][a] = ca[a];
        } else if (child == 1) {
          B[0][a] = ab[a];
          B[2][a] = bc[a];
        } else if (child == 2) {
          B[0][a] = ca[a];
          B[1][a] = bc[a];
        } else {
          B[0][a] = ab[a];
          B[1][a] = bc[a];
          B[2][a] = ca[a];
        }
      }
    }
    for (int q = 0; q < 3; ++q) {
      R beta[3], d[3];
      for (int a = 0; a < 3; ++a) {
        beta[a] = 0;
        for (int c = 0; c < 3; ++c) beta[a] += (c == q ? R(2) / R(3) : R(1) / R(6)) * B[c][a];
      }
      for (int dd = 0; dd < 3; ++dd)
        d[dd] = beta[0] * t.v[0][dd] + beta[1] * t.v[1][dd] + beta[2] * t.v[2][dd] - x[dd];
      cpx<R> G, F, H;
      R rr;
      ghfr(d[0], d[1], d[2], k, G, F, H, rr);
      const R dn = d[0] * t.n[0] + d[1] * t.n[1] + d[2] * t.n[2];
      if (kd) {
        const R wr = sign * w * rr, wk = -sign * w * k * dn;
        kd[0] = kd[0] + cmk(-wr * G.im, wr * G.re);
        kd[1] = kd[1] + wk * G;
      }
      const cpx<R> a = cy * F - dn * (cx * H);
      const cpx<R> b = cx * F;
      for (int dd = 0; dd < 3; ++dd) {
        const R pg = w * (a.re * d[dd] - b.re * t.n[dd]);
        tl[dd] -= pg;
        for (int c = 0; c < 3; ++c) g9l[3 * c + dd] += beta[c] * pg;
        gN[dd] -= w * b.re * d[dd];
      }
      gA += (cy * G - dn * (cx * F)).re;
    }
  }
  map_area_normal(t, gA * w / t.area, gN, g9l);
  for (int m = 0; m < 9; ++m) g9[m] += sign * g9l[m];
  for (int dd = 0; dd < 3; ++dd) tgt[dd] += sign * tl[dd];
}

__constant__ double c_vgl_x[32];
__constant__ double c_vgl_w[32];

// m0 = int_0^1 exp(i a s) ds = (exp(ia) - 1)/(ia) and m1 = int_0^1 s exp(i a s) ds
// = exp(ia)/(ia) + (exp(ia) - 1)/a^2, given sn = sin a, cs = cos a; below
// |a| = 0.5 by their power series sum_n (ia)^n / n! / (n + 1) and / (n + 2)
__device__ void moments01(double a, double sn, double cs, zd& m0, zd& m1) {
  if (fabs(a) < 0.5) {
    zd a0 = cmk(0.0, 0.0), a1 = a0, term = cmk(1.0, 0.0);  // (ia)^n / n!
#pragma unroll
    for (int n = 0; n < 30; ++n) {  // unrolled: the reciprocals fold to constants
      a0 = a0 + (1.0 / (n + 1.0)) * term;
      a1 = a1 + (1.0 / (n + 2.0)) * term;
      term = (1.0 / (n + 1.0)) * (term * cmk(0.0, a));
    }
    m0 = a0;
    m1 = a1;
    return;
  }
  const double ia = 1.0 / a, ia2 = ia * ia;
  m0 = cmk(sn * ia, (1.0 - cs) * ia);
  m1 = cmk(sn * ia + (cs - 1.0) * ia2, -cs * ia + sn * ia2);
}

// d/dV of Re(cy S_ii) for the exact self term (closed radial form, file
// header), the 32 Gauss-Legendre points of every panel split over the lanes of
// a warp; every lane returns the warp's sum in g9 (added).  With dks non-null
// the same points give dS_ii/dk = (1/4 pi) sum_edges int R^2 i m1(k R) dphi
// (m1 = int_0^1 s exp(i k R s) ds), returned in *dks on every lane.
__device__ void self_grad(const VTri& t, double k, zd cy, int lane, double* g9, zd* dks = nullptr) {
  double gl[3][3];  // grad lambda_a = (e_a x n) / (2A), e_a = V_{a+1} - V_{a+2}
  double dA[3][3];  // dA/dV_a = (1/2) e_a x n
  for (int a = 0; a < 3; ++a) {
    const double* b = t.v[(a + 1) % 3];
    const double* c = t.v[(a + 2) % 3];
    double e[3] = {b[0] - c[0], b[1] - c[1], b[2] - c[2]}, en[3];
    cross(e, t.n, en);
    for (int d = 0; d < 3; ++d) {
      gl[a][d] = en[d] / (2.0 * t.area);
      dA[a][d] = 0.5 * en[d];
    }
  }
  zd S = cmk(0.0, 0.0), SK = cmk(0.0, 0.0);
  zd J[3][3];
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) J[a][d] = cmk(0.0, 0.0);
  const double xq = c_vgl_x[lane], wgl = c_vgl_w[lane];
  for (int e = 0; e < 3; ++e) {
    const double* a = t.v[e];
    const double* b = t.v[(e + 1) % 3];
    double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double len = sqrt(ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2]);
    double tv[3] = {ab[0] / len, ab[1] / len, ab[2] / len};
    double xa[3] = {t.c[0] - a[0], t.c[1] - a[1], t.c[2] - a[2]};
    double pr = xa[0] * tv[0] + xa[1] * tv[1] + xa[2] * tv[2];
    double fx[3] = {xa[0] - pr * tv[0], xa[1] - pr * tv[1], xa[2] - pr * tv[2]};
    double dist = sqrt(fx[0] * fx[0] + fx[1] * fx[1] + fx[2] * fx[2]);
    double fh[3] = {-fx[0] / dist, -fx[1] / dist, -fx[2] / dist};  // centroid -> foot of the edge
    const double u0 = asinh(-pr / dist), u1 = asinh((len - pr) / dist);
    // the direction's tanh(u) has poles at u = +-i pi/2: panels of length <= 4
    // keep 32-point Gauss-Legendre at rounding level on slivers, whose u-range
    // grows like 2 log(edge / height)
    const int npan = max(1, (int)ceil((u1 - u0) / 4.0));
    const double plen = (u1 - u0) / npan;
    const double half = 0.5 * plen;
    for (int pn = 0; pn < npan; ++pn) {
      const double u = u0 + plen * (pn + 0.5) + half * xq;
      // cosh and sinh from one exponential, and one reciprocal of cosh
      const double eu = exp(u), ieu = 1.0 / eu;
      const double ch = 0.5 * (eu + ieu), sh = 0.5 * (eu - ieu), ich = 1.0 / ch;
      const double R = dist * ch;
      const double wq = half * wgl * ich;  // d phi = du / cosh(u)
      double sn, cs;
      sincos(k * R, &sn, &cs);
      zd m0, m1;
      moments01(k * R, sn, cs, m0, m1);
      S = S + (wq * R) * m0;
      SK = SK + (wq * R * R) * cmk(-m1.im, m1.re);  // i R^2 m1
      const zd K = R * (cmk(cs, sn) - 2.0 * m0);
      double dir[3];
      for (int d = 0; d < 3; ++d) dir[d] = (fh[d] + sh * tv[d]) * ich;
      for (int va = 0; va < 3; ++va) {
        const double s = dir[0] * gl[va][0] + dir[1] * gl[va][1] + dir[2] * gl[va][2];
        for (int d = 0; d < 3; ++d) J[va][d] = J[va][d] + (wq * s * dir[d]) * K;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    S.re += __shfl_xor_sync(0xffffffffu, S.re, o);
    S.im += __shfl_xor_sync(0xffffffffu, S.im, o);
    SK.re += __shfl_xor_sync(0xffffffffu, SK.re, o);
    SK.im += __shfl_xor_sync(0xffffffffu, SK.im, o);
    for (int va = 0; va < 3; ++va)
      for (int d = 0; d < 3; ++d) {
        J[va][d].re += __shfl_xor_sync(0xffffffffu, J[va][d].re, o);
        J[va][d].im += __shfl_xor_sync(0xffffffffu, J[va][d].im, o);
      }
  }
  const double c4 = 1.0 / (4.0 * BEM_PI);
  for (int va = 0; va < 3; ++va)
    for (int d = 0; d < 3; ++d) {
      const zd dS = (c4 * dA[va][d] / t.area) * S + c4 * J[va][d];
      g9[3 * va + d] += (cy * dS).re;
    }
  if (dks) *dks = c4 * SK;
}

// One warp per row i of the correction matrix: for every non-self (i, j) the
// refined rule minus R_0 (the self pairs are k_gv_self's); with dk non-null
// the same points give the pair's d/dk of (refined rule - R_0), added to *dk
// as Re((dS/dk) cy - (dD/dk) cx).  Launched with 128 threads.  Collocation-point
// gradients are summed over the warp into gx; vertex gradients of Gamma_j go
// to gel[j] (9 doubles: V_0, V_1, V_2).  With f32 (mixed modes) the non-self
// pairs run in FP32 with the triangle relative to the collocation point.
__global__ void k_gv_corr(int64_t nt, int nrhs, int f32, double k, const double* __restrict__ cent,
                          const double* __restrict__ qpt, const double* __restrict__ nrm,
                          const double* __restrict__ area, const double* __restrict__ hmax,
                          const int* __restrict__ ptr, const int* __restrict__ col, const double4* __restrict__ yx,
                          const double2* __restrict__ gs, double* __restrict__ gx, double* __restrict__ gel,
                          double* __restrict__ dk) {
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  double tg[3] = {0.0, 0.0, 0.0};
  double dkp = 0.0;  // Re((dS/dk) cy - (dD/dk) cx) of the row's corrections, with dk
  if (i < nt) {
    const double x[3] = {cent[3 * i], cent[3 * i + 1], cent[3 * i + 2]};
    for (int e = ptr[i] + lane; e < ptr[i + 1]; e += 32) {
      const int64_t j = col[e];
      if (j == i) continue;  // the self pair: k_gv_self
      VTri t;
      vload(qpt, nrm, cent, area, hmax, j, t);
      const double dd[3] = {t.c[0] - x[0], t.c[1] - x[1], t.c[2] - x[2]};
      const double dist = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
      const int L = dist < 2.0 * t.h ? 2 : (dist < 4.0 * t.h ? 1 : 0);
      if (L == 0) continue;  // the rules agree: no correction
      zd cy = cmk(0.0, 0.0), cx = cmk(0.0, 0.0);
      for (int r = 0; r < nrhs; ++r) {
        const double2 g = gs[(int64_t)r * nt + i];
        const double4 v = yx[(int64_t)r * nt + j];
        const zd cg = cmk(g.x, -g.y);
        cy = cy + cg * cmk(v.x, v.y);
        cx = cx + cg * cmk(v.z, v.w);
      }
      double g9[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, tt[3] = {0, 0, 0};
      if (f32) {
        // mixed modes: both rules of a non-self pair in FP32, the triangle
        // relative to the collocation point (as the correction values were built)
        VTriT<float> tf;
        for (int a = 0; a < 3; ++a)
          for (int d = 0; d < 3; ++d) tf.v[a][d] = (float)(t.v[a][d] - x[d]);
        for (int d = 0; d < 3; ++d) {
          tf.n[d] = (float)t.n[d];
          tf.c[d] = (float)(t.c[d] - x[d]);
        }
        tf.area = (float)t.area;
        tf.h = (float)t.h;
        const float x0[3] = {0.f, 0.f, 0.f};
        const cpx<float> cyf = cmk((float)cy.re, (float)cy.im), cxf = cmk((float)cx.re, (float)cx.im);
        float g9f[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, ttf[3] = {0, 0, 0};
        cpx<float> kd[2] = {cmk(0.f, 0.f), cmk(0.f, 0.f)};
        rule_grad(x0, tf, 0, (float)k, cyf, cxf, -1.0f, ttf, g9f, dk ? kd : nullptr);
        rule_grad(x0, tf, L, (float)k, cyf, cxf, 1.0f, ttf, g9f, dk ? kd : nullptr);
        dkp += (double)kd[0].re * cy.re - (double)kd[0].im * cy.im - ((double)kd[1].re * cx.re - (double)kd[1].im * cx.im);
        for (int d = 0; d < 3; ++d) tg[d] += (double)ttf[d];
        for (int m = 0; m < 9; ++m) atomicAdd(&gel[9 * j + m], (double)g9f[m]);
        continue;
      }
      zd kd[2] = {cmk(0.0, 0.0), cmk(0.0, 0.0)};
      rule_grad(x, t, 0, k, cy, cx, -1.0, tt, g9, dk ? kd : nullptr);
      rule_grad(x, t, L, k, cy, cx, 1.0, tt, g9, dk ? kd : nullptr);
      dkp += (kd[0] * cy).re - (kd[1] * cx).re;
      for (int d = 0; d < 3; ++d) tg[d] += tt[d];
      for (int m = 0; m < 9; ++m) atomicAdd(&gel[9 * j + m], g9[m]);
    }
  }
  for (int d = 0; d < 3; ++d)
    for (int o = 16; o > 0; o >>= 1) tg[d] += __shfl_xor_sync(0xffffffffu, tg[d], o);
  if (i < nt && lane == 0)
    for (int d = 0; d < 3; ++d) atomicAdd(&gx[3 * i + d], tg[d]);
  if (dk) {
    // one atomic add per block of four rows
    for (int o = 16; o > 0; o >>= 1) dkp += __shfl_xor_sync(0xffffffffu, dkp, o);
    __shared__ double s_dk[4];
    if (lane == 0) s_dk[threadIdx.x >> 5] = dkp;
    __syncthreads();
    if (threadIdx.x == 0) {
      const double sum = s_dk[0] + s_dk[1] + s_dk[2] + s_dk[3];
      if (sum != 0.0) atomicAdd(dk, sum);
    }
  }
}

// the self pairs, one warp per element (the lanes split the Gauss-Legendre
// points of the exact term): the exact self term's vertex gradient minus
// R_0's, and R_0's collocation gradient spread over the element's own vertices
// (its centroid is the collocation point).  Runs after k_gv_corr, so gel[j] is
// updated in place.  With dk non-null the same quadrature gives the self
// pair's d/dk of (exact - R_0), added to *dk.  Launched with 128 threads.
__global__ void __launch_bounds__(128) k_gv_self(int64_t nt, int nrhs, double k, const double* __restrict__ cent,
                                                 const double* __restrict__ qpt, const double* __restrict__ nrm,
                                                 const double* __restrict__ area, const double* __restrict__ hmax,
                                                 const double4* __restrict__ yx, const double2* __restrict__ gs,
                                                 double* __restrict__ gel, double* __restrict__ dk) {
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  double part = 0.0;  // Re((dS_ii/dk - R_0's) cy - (-R_0's dD/dk) cx), with dk
  if (i < nt) {  // the whole warp: i is the same on every lane
    VTri t;
    vload(qpt, nrm, cent, area, hmax, i, t);
    const double x[3] = {t.c[0], t.c[1], t.c[2]};
    zd cy = cmk(0.0, 0.0), cx = cmk(0.0, 0.0);
    for (int r = 0; r < nrhs; ++r) {
      const double2 g = gs[(int64_t)r * nt + i];
      const double4 v = yx[(int64_t)r * nt + i];
      const zd cg = cmk(g.x, -g.y);
      cy = cy + cg * cmk(v.x, v.y);
      cx = cx + cg * cmk(v.z, v.w);
    }
    double g9[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, tt[3] = {0, 0, 0};
    zd dks = cmk(0.0, 0.0);
    self_grad(t, k, cy, lane, g9, dk ? &dks : nullptr);
    if (lane == 0) {
      zd kd[2] = {cmk(0.0, 0.0), cmk(0.0, 0.0)};
      rule_grad(x, t, 0, k, cy, cx, -1.0, tt, g9, dk ? kd : nullptr);  // kd = (-s0, -d0)
      for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 3; ++d) g9[3 * a + d] += tt[d] / 3.0;
      for (int m = 0; m < 9; ++m) gel[9 * i + m] += g9[m];
      part = ((dks + kd[0]) * cy).re - (kd[1] * cx).re;
    }
  }
  if (dk) {
    // one atomic add per block of four elements
    __shared__ double s_dk[4];
    if (lane == 0) s_dk[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      const double sum = s_dk[0] + s_dk[1] + s_dk[2] + s_dk[3];
      if (sum != 0.0) atomicAdd(dk, sum);
    }
  }
}

// Per element: regular-rule point, area and normal gradients and the
// collocation-point gradient mapped onto the three vertices, plus the
// corrections; added into the caller's vertex order.
__global__ void k_gv_finish(int64_t nt, const double* __restrict__ cent, const double* __restrict__ qpt,
                            const double* __restrict__ nrm, const double* __restrict__ area,
                            const double* __restrict__ hmax, const int* __restrict__ tri,
                            const double* __restrict__ gx, const double* __restrict__ gq,
                            const double* __restrict__ ga, const double* __restrict__ gn,
                            const double* __restrict__ gel, double* __restrict__ dV) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= nt) return;
  VTri t;
  vload(qpt, nrm, cent, area, hmax, j, t);
  double g9[9];
  for (int m = 0; m < 9; ++m) g9[m] = gel[9 * j + m];
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) {
      double s = gx[3 * j + d] / 3.0;
      for (int q = 0; q < 3; ++q) s += (q == a ? 2.0 / 3.0 : 1.0 / 6.0) * gq[9 * j + 3 * q + d];
      g9[3 * a + d] += s;
    }
  const double gN[3] = {gn[3 * j], gn[3 * j + 1], gn[3 * j + 2]};
  map_area_normal(t, ga[j], gN, g9);
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) atomicAdd(&dV[3 * (int64_t)tri[3 * j + a] + d], g9[3 * a + d]);
}

// ------------------------------------------------- regular rule by the tree --
// The regular-rule sums of the two passes above are fields, so the octree
// evaluates them in O(N log N):
//   target side  T_i = grad_x z(x_i), z = S y - D x under R_0 over every pair:
//                the walk of the off-surface evaluation at the centroids, its
//                near leaves summed with R_0 (no refined rules);
//   source side  with psi(y) = sum_i conj(g_i) G(y - x_i) (point charges at
//                the centroids): PS = grad psi, Fs n + QH = (Hess psi) n,
//                GS = psi, GD = n.grad psi at every quadrature point: the
//                multipoles of the charges (from the L2P rows, which hold
//                R~(x_i - c) of every centroid), M2M, and a walk at the
//                quadrature points whose far boxes run the M2P with the point
//                moved along n as a dual number, near leaves summed directly.

// weighted densities (wgt y, wgt x) in tree order from the gradient's FP64 copy
template <typename V4>
__global__ void k_gvf_dens(int64_t nt, int nrhs, const double* __restrict__ wgt, const double4* __restrict__ yx,
                           V4* __restrict__ dens) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nt) return;
  const double w = wgt[s];
  for (int r = 0; r < nrhs; ++r) {
    const double4 v = yx[(int64_t)r * nt + s];
    V4 d;
    d.x = w * v.x;
    d.y = w * v.y;
    d.z = w * v.z;
    d.w = w * v.w;
    dens[(int64_t)r * nt + s] = d;
  }
}

// gx_j += sum_r Re(conj(g_j) grad z(x_j)) from the walk's sums (point i of the
// walk is centroid perm[i])
__global__ void k_gvf_tgt_out(int64_t nt, int nrhs, const int* __restrict__ perm, const double* __restrict__ acc,
                              const double2* __restrict__ gs, double* __restrict__ gx) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nt) return;
  const int64_t j = perm[i];
  double t[3] = {0.0, 0.0, 0.0};
  for (int r = 0; r < nrhs; ++r) {
    const double2 g = gs[(int64_t)r * nt + j];
    const double* a = acc + 6 * ((int64_t)r * nt + i);
    for (int d = 0; d < 3; ++d) t[d] += g.x * a[2 * d] + g.y * a[2 * d + 1];
  }
  for (int d = 0; d < 3; ++d) gx[3 * j + d] += t[d];
}

// Multipoles of the point charges conj(g_j) at the centroids of one leaf (one
// block per leaf and right-hand side, threads over the coefficients):
// M~_e = i k sum_j conj(g_j) conj(R~_e(x_j - c)), the normalisation of the
// P2M rows (4 pi i k conj(R~) against densities that carry 1 / (4 pi)).
template <typename R>
__global__ void k_gvf_p2m(const int* __restrict__ leafbox, int64_t nt, int P, const int* __restrict__ bstart,
                          const int* __restrict__ bend, const int64_t* __restrict__ row_off,
                          const R* __restrict__ rows_r, const double2* __restrict__ gs, double k, int64_t exp_base,
                          int64_t exp_stride, R* __restrict__ M) {
  const int b = leafbox[blockIdx.x], r = blockIdx.y;
  const double2* gr = gs + (int64_t)r * nt;
  for (int e = threadIdx.x; e < P; e += blockDim.x) {
    R are = 0, aim = 0;
    for (int j = bstart[b]; j < bend[b]; ++j) {
      const R* row = rows_r + 2 * row_off[j];
      const R rr = row[2 * e], ri = row[2 * e + 1];
      const double2 g = gr[j];
      const R gx = (R)g.x, gy = (R)g.y;
      // conj(g) conj(row) = (gx rr - gy ri) - i (gx ri + gy rr)
      are += gx * rr - gy * ri;
      aim -= gx * ri + gy * rr;
    }
    R* out = M + 2 * ((int64_t)r * exp_stride + exp_base + (int64_t)b * P + e);
    out[0] = (R)(-k) * aim;
    out[1] = (R)k * are;
  }
}

// Near leaves, one thread per walk point: consecutive walk points are
// neighbours along the Morton curve, so the lanes of a warp walk nearly the
// same leaves and read the same elements.  In FP32 the coordinates of every
// element are held relative to its leaf's centre as high and low FP32 parts
// (GvRec), and the leaf's offset from the point the same way, so that a
// separation (hi + off_hi) + (lo + off_lo) keeps FP32 relative accuracy for
// the closest pairs (an element's own quadrature points and centroid).
struct GvRec {
  float qh[9], ql[9];  // quadrature points - leaf centre
  float ch[3], cl[3];  // centroid - leaf centre
  float n[3], w;       // unit normal, area / 3
};

__global__ void k_gvf_split(int64_t nt, const int* __restrict__ leaf_of, const unsigned char* __restrict__ leaf_lev,
                            WalkTree wt, const double* __restrict__ cent, const double* __restrict__ qpt,
                            const double* __restrict__ nrm, const double* __restrict__ area, GvRec* __restrict__ rec) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nt) return;
  const double* c = wt.lv[leaf_lev[e]].centre + 3 * (int64_t)leaf_of[e];
  GvRec g;
  for (int m = 0; m < 9; ++m) {
    const double v = qpt[9 * e + m] - c[m % 3];
    g.qh[m] = (float)v;
    g.ql[m] = (float)(v - (double)g.qh[m]);
  }
  for (int d = 0; d < 3; ++d) {
    const double v = cent[3 * e + d] - c[d];
    g.ch[d] = (float)v;
    g.cl[d] = (float)(v - (double)g.ch[d]);
    g.n[d] = (float)nrm[3 * e + d];
  }
  g.w = (float)(area[e] / 3.0);
  rec[e] = g;
}

// sum over the lanes of a team (team consecutive lanes, a power of two)
template <typename R, int NV>
__device__ __forceinline__ void gv_team_sum(R (&v)[NV], int team) {
  for (int o = team >> 1; o > 0; o >>= 1)
#pragma unroll
    for (int c = 0; c < NV; ++c) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
}

// the leaf's offset from X: FP64 for R = double, FP32 high and low parts otherwise
template <typename R>
struct LeafOff {
  R h[3], l[3];
  __device__ __forceinline__ LeafOff(const double* c, const double* X) {
    for (int d = 0; d < 3; ++d) {
      const double v = c[d] - X[d];
      h[d] = (R)v;
      l[d] = (R)(v - (double)h[d]);
    }
  }
};

// Target side near leaves (R_0 over every element of every near leaf, the
// point's own element included): adds grad_x z to acc[r][i][0..2].  A team
// of lanes per point walks the tree together and strides over each leaf's
// elements.
template <typename R, int NR>
__global__ void __launch_bounds__(128) k_gvf_tnear(int r0, int team, int64_t nt, WalkTree wt, double k, int64_t np,
                                                   const double* __restrict__ pts, const int* __restrict__ tcs,
                                                   const GvRec* __restrict__ rec, const double* __restrict__ qpt,
                                                   const double* __restrict__ nrm, const double* __restrict__ area,
                                                   const double4* __restrict__ yx, double* __restrict__ acc) {
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t i = gt / team;
  const int tl = (int)(gt & (team - 1));
  const bool live = i < np;
  const R kk = (R)k;
  R T[NR * 6];
#pragma unroll
  for (int c = 0; c < NR * 6; ++c) T[c] = 0;
  if (live) {
    const double X[3] = {pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]};
    const int t[3] = {tcs[3 * i], tcs[3 * i + 1], tcs[3 * i + 2]};
    tree_walk(wt, t, [&](int kind, int l, int b) {
      if (kind != 1) return;
      const LeafOff<R> off(wt.lv[l].centre + 3 * b, X);
      const int e1 = wt.lv[l].end[b];
      for (int j = wt.lv[l].start[b] + tl; j < e1; j += team) {
        R n[3], w;
        R y[9];
        if constexpr (sizeof(R) == 4) {
          const GvRec& g = rec[j];
#pragma unroll
          for (int m = 0; m < 9; ++m) y[m] = (g.qh[m] + off.h[m % 3]) + (g.ql[m] + off.l[m % 3]);
#pragma unroll
          for (int d = 0; d < 3; ++d) n[d] = g.n[d];
          w = g.w;
        } else {
#pragma unroll
          for (int m = 0; m < 9; ++m) y[m] = qpt[9 * (int64_t)j + m] - X[m % 3];
#pragma unroll
          for (int d = 0; d < 3; ++d) n[d] = nrm[3 * (int64_t)j + d];
          w = area[j] / 3.0;
        }
        cpx<R> wy[NR], wx[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          const double4 v = yx[(int64_t)(r0 + q) * nt + j];
          wy[q] = cmk((R)v.x * w, (R)v.y * w);
          wx[q] = cmk((R)v.z * w, (R)v.w * w);
        }
#pragma unroll
        for (int qp = 0; qp < 3; ++qp) {
          const R d0 = y[3 * qp], d1 = y[3 * qp + 1], d2 = y[3 * qp + 2];
          cpx<R> G, F, H;
          ghf(d0, d1, d2, kk, G, F, H);
          const R dn = d0 * n[0] + d1 * n[1] + d2 * n[2];
#pragma unroll
          for (int q = 0; q < NR; ++q) {
            const cpx<R> a = dn * (H * wx[q]) - F * wy[q];
            const cpx<R> bb = F * wx[q];
            T[6 * q] += d0 * a.re + n[0] * bb.re;
            T[6 * q + 1] += d0 * a.im + n[0] * bb.im;
            T[6 * q + 2] += d1 * a.re + n[1] * bb.re;
            T[6 * q + 3] += d1 * a.im + n[1] * bb.im;
            T[6 * q + 4] += d2 * a.re + n[2] * bb.re;
            T[6 * q + 5] += d2 * a.im + n[2] * bb.im;
          }
        }
      }
    });
  }
  gv_team_sum(T, team);
  if (!live || tl != 0) return;
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    double* o = acc + 6 * ((int64_t)(r0 + q) * np + i);
#pragma unroll
    for (int c = 0; c < 6; ++c) o[c] += (double)T[6 * q + c];
  }
}

// Source side near leaves: the point charges conj(g_e) at the centroids of
// every near leaf, at the quadrature point i of element perm[i] / 3; adds
// (psi, grad psi, n.grad psi, (Hess psi) n) to acc[r][i][0..7].  Teams of
// lanes as in k_gvf_tnear.
template <typename R, int NR>
__global__ void __launch_bounds__(128) k_gvf_snear(int r0, int team, int64_t nt, WalkTree wt, double k, int64_t np,
                                                   const double* __restrict__ pts, const int* __restrict__ tcs,
                                                   const int* __restrict__ perm, const GvRec* __restrict__ rec,
                                                   const double* __restrict__ cent, const double* __restrict__ nrm,
                                                   const double2* __restrict__ gs, double* __restrict__ acc) {
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t i = gt / team;
  const int tl = (int)(gt & (team - 1));
  const bool live = i < np;
  const R kk = (R)k;
  R sm[NR * 16];
#pragma unroll
  for (int c = 0; c < NR * 16; ++c) sm[c] = 0;
  if (live) {
    const double X[3] = {pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]};
    const int t[3] = {tcs[3 * i], tcs[3 * i + 1], tcs[3 * i + 2]};
    const int64_t jq = perm[i] / 3;
    const R n0 = (R)nrm[3 * jq], n1 = (R)nrm[3 * jq + 1], n2 = (R)nrm[3 * jq + 2];
    tree_walk(wt, t, [&](int kind, int l, int b) {
      if (kind != 1) return;
      const LeafOff<R> off(wt.lv[l].centre + 3 * b, X);
      const int e1 = wt.lv[l].end[b];
      for (int e = wt.lv[l].start[b] + tl; e < e1; e += team) {
        // d = X - x_e
        R d0, d1, d2;
        if constexpr (sizeof(R) == 4) {
          const GvRec& g = rec[e];
          d0 = -((g.ch[0] + off.h[0]) + (g.cl[0] + off.l[0]));
          d1 = -((g.ch[1] + off.h[1]) + (g.cl[1] + off.l[1]));
          d2 = -((g.ch[2] + off.h[2]) + (g.cl[2] + off.l[2]));
        } else {
          d0 = X[0] - cent[3 * (int64_t)e];
          d1 = X[1] - cent[3 * (int64_t)e + 1];
          d2 = X[2] - cent[3 * (int64_t)e + 2];
        }
        cpx<R> G, F, H;
        ghf(d0, d1, d2, kk, G, F, H);
        const R dn = d0 * n0 + d1 * n1 + d2 * n2;
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          const double2 g = gs[(int64_t)(r0 + q) * nt + e];
          const cpx<R> c = cmk((R)g.x, (R)(-g.y));
          const cpx<R> cF = c * F, cG = c * G, cH = dn * (c * H);
          R* a = sm + 16 * q;
          a[0] += cG.re;
          a[1] += cG.im;
          a[2] += d0 * cF.re;
          a[3] += d0 * cF.im;
          a[4] += d1 * cF.re;
          a[5] += d1 * cF.im;
          a[6] += d2 * cF.re;
          a[7] += d2 * cF.im;
          a[8] += dn * cF.re;
          a[9] += dn * cF.im;
          a[10] += d0 * cH.re + n0 * cF.re;
          a[11] += d0 * cH.im + n0 * cF.im;
          a[12] += d1 * cH.re + n1 * cF.re;
          a[13] += d1 * cH.im + n1 * cF.im;
          a[14] += d2 * cH.re + n2 * cF.re;
          a[15] += d2 * cH.im + n2 * cF.im;
        }
      }
    });
  }
  gv_team_sum(sm, team);
  if (!live || tl != 0) return;
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    double* a = acc + 16 * ((int64_t)(r0 + q) * np + i);
#pragma unroll
    for (int c = 0; c < 16; ++c) a[c] += (double)sm[16 * q + c];
  }
}

// the source side's sums at walk point i (quadrature point p = perm[i] of
// element j = p / 3) into the point, area and normal gradients, as the
// source-major pass leaves them
__global__ void k_gvf_src_out(int64_t np, int nrhs, int64_t nt, const int* __restrict__ perm,
                              const double* __restrict__ acc, const double* __restrict__ area,
                              const double4* __restrict__ yx, double* __restrict__ gq, double* __restrict__ ga,
                              double* __restrict__ gn) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int64_t p = perm[i], j = p / 3;
  const double w = area[j] / 3.0;
  double tq[3] = {0, 0, 0}, tn[3] = {0, 0, 0}, ta = 0;
  for (int r = 0; r < nrhs; ++r) {
    const double* a = acc + 16 * ((int64_t)r * np + i);
    const double4 v = yx[(int64_t)r * nt + j];
    const zd yj = cmk(v.x, v.y), xj = cmk(v.z, v.w);
    for (int d = 0; d < 3; ++d) {
      const zd ps = cmk(a[2 + 2 * d], a[3 + 2 * d]), qh = cmk(a[10 + 2 * d], a[11 + 2 * d]);
      tq[d] += (yj * ps - xj * qh).re;
      tn[d] -= (xj * ps).re;
    }
    ta += (yj * cmk(a[0], a[1]) - xj * cmk(a[8], a[9])).re;
  }
  for (int d = 0; d < 3; ++d) {
    gq[3 * p + d] += w * tq[d];
    atomicAdd(&gn[3 * j + d], w * tn[d]);
  }
  atomicAdd(&ga[j], ta / 3.0);
}

template <typename R>
static int grad_tree_impl(bem_handle* h, int nrhs, const double4* yx, const double2* gs, double* gx, double* gq,
                          double* ga, double* gn, cudaStream_t s) {
  typedef typename std::conditional<sizeof(R) == 4, float4, double4>::type V4;
  const int64_t nt = h->nt, nq = 3 * nt;
  // R_0 everywhere: a far box only needs a convergent multipole at the point,
  // so the gap asked for is one longest edge of the box (not the four that
  // keep refined-rule pairs out of the off-surface walk's far boxes)
  WalkTree wt = bem_walk_tree(h);
  wt.gap_scale2 = 1.0f / 16.0f;
  int nl = 0;
  WalkOrder wo;
  double* acc = nullptr;
  GvRec* rec = nullptr;
  int rc = BEM_OK;
  auto cu = [&](cudaError_t e) {
    if (rc == BEM_OK && e != cudaSuccess)
      rc = bem_fail(e == cudaErrorMemoryAllocation ? BEM_ERR_OOM : BEM_ERR_CUDA, cudaGetErrorString(e));
    return rc != BEM_OK;
  };
  // lanes per walk point: enough that the points fill every SM about twice
  auto team_of = [&](int64_t np) {
    int tm = 1;
    while (tm < 32 && np * tm < (int64_t)h->nsm * 4096) tm <<= 1;
    return tm;
  };
  // right-hand sides in chunks of 4, then 2, then 1
  auto by_chunks = [&](int n, auto&& f) {
    for (int r0 = 0; r0 < n && rc == BEM_OK;) {
      const int rem = n - r0;
      if (rem >= 4) {
        f(std::integral_constant<int, 4>(), r0);
        r0 += 4;
      } else if (rem >= 2) {
        f(std::integral_constant<int, 2>(), r0);
        r0 += 2;
      } else {
        f(std::integral_constant<int, 1>(), r0);
        r0 += 1;
      }
    }
  };
  do {
    if (cu(cudaMallocAsync((void**)&acc, 16 * sizeof(double) * nq * nrhs, s))) break;
    // target side: grad z at the centroids, z from the operator's own multipoles
    k_gvf_dens<V4><<<nblk(nt, 256), 256, 0, s>>>(nt, nrhs, h->wgt, yx, (V4*)h->dens);
    if (cu(cudaGetLastError())) break;
    if ((rc = bem_run_upward(h, nrhs, s)) != BEM_OK) break;
    if (sizeof(R) == 4) {
      if (cu(cudaMallocAsync((void**)&rec, sizeof(GvRec) * nt, s))) break;
      k_gvf_split<<<nblk(nt, 128), 128, 0, s>>>(nt, h->leaf_of, h->leaf_lev, wt, h->cent, h->qpt, h->nrm,
                                                h->area, rec);
      if (cu(cudaGetLastError())) break;
    }
    if ((rc = bem_walk_order(wt, nt, h->cent, wo, s)) != BEM_OK) break;
    if ((rc = bem_evf_far(h, wt, nrhs, 1, nt, wo.spts, wo.tcs, acc, wo.nearflag, team_of(nt), s)) != BEM_OK) break;
    by_chunks(nrhs, [&](auto nr, int r0) {
      const int tm = team_of(nt);
      k_gvf_tnear<R, decltype(nr)::value><<<nblk(nt * tm, 128), 128, 0, s>>>(r0, tm, nt, wt, h->k, nt, wo.spts,
                                                                             wo.tcs, rec, h->qpt, h->nrm, h->area,
                                                                             yx, acc);
      cu(cudaGetLastError());
    });
    if (rc != BEM_OK) break;
    k_gvf_tgt_out<<<nblk(nt, 256), 256, 0, s>>>(nt, nrhs, wo.perm, acc, gs, gx);
    if (cu(cudaGetLastError())) break;
    bem_walk_free(wo, s);
    // source side: multipoles of the charges conj(g) at the centroids
    if (cu(cudaMemsetAsync(h->Mexp, 0, 2 * sizeof(R) * h->exp_total * nrhs, s))) break;
    for (int l = 2; l <= h->L && rc == BEM_OK; ++l) {
      const LevelInfo& lf = h->lev[l];
      if (lf.nleaf == 0) continue;
      k_gvf_p2m<R><<<dim3(lf.nleaf, nrhs), 128, 0, s>>>(lf.leafbox, nt, lf.P, lf.start, lf.end, h->row_off,
                                                        (const R*)h->l2p_rows, gs, h->k, lf.exp_base, h->exp_total,
                                                        (R*)h->Mexp);
      cu(cudaGetLastError());
    }
    if (rc != BEM_OK) break;
    for (int l = h->L - 1; l >= 2 && rc == BEM_OK; --l)
      rc = bem_run_grouped(h, h->m2m[l], h->Mexp, h->Mexp, nrhs, s, &nl);
    if (rc != BEM_OK) break;
    if ((rc = bem_walk_order(wt, nq, h->qpt, wo, s)) != BEM_OK) break;
    if ((rc = bem_gvf_far(h, wt, nrhs, nq, wo.spts, wo.tcs, wo.perm, team_of(nq), acc, s)) != BEM_OK) break;
    by_chunks(nrhs, [&](auto nr, int r0) {
      const int tm = team_of(nq);
      k_gvf_snear<R, decltype(nr)::value><<<nblk(nq * tm, 128), 128, 0, s>>>(r0, tm, nt, wt, h->k, nq, wo.spts,
                                                                             wo.tcs, wo.perm, rec, h->cent, h->nrm,
                                                                             gs, acc);
      cu(cudaGetLastError());
    });
    if (rc != BEM_OK) break;
    k_gvf_src_out<<<nblk(nq, 256), 256, 0, s>>>(nq, nrhs, nt, wo.perm, acc, h->area, yx, gq, ga, gn);
    cu(cudaGetLastError());
  } while (false);
  if (acc) cudaFreeAsync(acc, s);
  if (rec) cudaFreeAsync(rec, s);
  bem_walk_free(wo, s);
  return rc;
}

int bem_grad_vertices(bem_handle* h, int nrhs, const double4* yx, const double2* gs, double* dvertices, double* dk,
                      cudaStream_t s) {
  const int64_t nt = h->nt, nv = h->nv;
  double *gx, *gq, *ga, *gn, *gel, *dV;
  const size_t nd = dvertices ? (size_t)nt * (3 + 9 + 1 + 3 + 9) + (size_t)nv * 3 : (size_t)nt * 3;
  double* buf;
  BEM_CUDA(cudaMallocAsync((void**)&buf, nd * sizeof(double), s));
  BEM_CUDA(cudaMemsetAsync(buf, 0, nd * sizeof(double), s));
  gx = buf;
  gq = gx + 3 * nt;
  ga = gq + 9 * nt;
  gn = ga + nt;
  gel = gn + 3 * nt;
  dV = gel + 9 * nt;
  const bool f64 = bem_is_fp64(h);
  // split the streamed range so that the grid fills the GPU several times
  // over: 128 targets (or quadrature points) per block leave too few blocks
  auto chunked = [&](const void* fn, int64_t rows, int64_t& chunk) {
    int res = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&res, fn, 128, 0);
    const int64_t base = (int64_t)nblk(rows, 128) * nrhs;
    const int64_t want = (int64_t)4 * h->nsm * max(res, 1);
    const int64_t tiles = (nt + 127) / 128;
    const int64_t nz = max((int64_t)1, min(tiles, (want + base - 1) / base));
    chunk = ((tiles + nz - 1) / nz) * 128;
    return dim3(nblk(rows, 128), nrhs, (unsigned)((nt + chunk - 1) / chunk));
  };
  // the regular rule through the tree on FMM handles (unless the all-pairs
  // sums are asked for); dL/dk's regular part stays an all-pairs sum
  const bool tree = dvertices && bem_is_fmm(h) && h->L >= 2 && !h->grad_direct;
  // the all-pairs target pass sums the centroid gradients only when the
  // vertices are asked for without the tree; otherwise dL/dk's part alone
  const bool gxpass = dvertices && !tree;
  int64_t ct = 0, cs = 0;
  if (gxpass || dk) {
    const void* ft = f64 ? (gxpass ? (const void*)k_gv_target<double, true> : (const void*)k_gv_target<double, false>)
                         : (gxpass ? (const void*)k_gv_target<float, true> : (const void*)k_gv_target<float, false>);
    const dim3 gt = chunked(ft, nt, ct);
#define GV_TARGET(RT, GXV) \
  k_gv_target<RT, GXV><<<gt, 128, 0, s>>>(nt, h->k, h->cent, h->qpt, h->nrm, h->area, yx, gs, ct, gx, dk)
    if (f64) {
      if (gxpass)
        GV_TARGET(double, true);
      else
        GV_TARGET(double, false);
    } else {
      if (gxpass)
        GV_TARGET(float, true);
      else
        GV_TARGET(float, false);
    }
#undef GV_TARGET
    BEM_CUDA(cudaGetLastError());
  }
  if (!dvertices) {
    // only the regular-rule part of dL/dk was asked for
    BEM_CUDA(cudaFreeAsync(buf, s));
    return BEM_OK;
  }
  if (tree) {
    BEM_TRY(f64 ? grad_tree_impl<double>(h, nrhs, yx, gs, gx, gq, ga, gn, s)
                : grad_tree_impl<float>(h, nrhs, yx, gs, gx, gq, ga, gn, s));
  } else {
    const void* fs = f64 ? (const void*)k_gv_source<double> : (const void*)k_gv_source<float>;
    const dim3 gsrc = chunked(fs, 3 * nt, cs);
    if (f64)
      k_gv_source<double><<<gsrc, 128, 0, s>>>(nt, h->k, h->cent, h->qpt, h->nrm, h->area, yx, gs, cs, gq, ga, gn);
    else
      k_gv_source<float><<<gsrc, 128, 0, s>>>(nt, h->k, h->cent, h->qpt, h->nrm, h->area, yx, gs, cs, gq, ga, gn);
  }
  BEM_CUDA(cudaGetLastError());
  double glx[32], glw[32];
  bem_gl_host(32, glx, glw);
  BEM_CUDA(cudaMemcpyToSymbolAsync(c_vgl_x, glx, sizeof(glx), 0, cudaMemcpyHostToDevice, s));
  BEM_CUDA(cudaMemcpyToSymbolAsync(c_vgl_w, glw, sizeof(glw), 0, cudaMemcpyHostToDevice, s));
  k_gv_corr<<<nblk(nt * 32, 128), 128, 0, s>>>(nt, nrhs, f64 ? 0 : 1, h->k, h->cent, h->qpt, h->nrm, h->area, h->hmax,
                                               h->corr_ptr, h->corr_col, yx, gs, gx, gel, dk);
  BEM_CUDA(cudaGetLastError());
  k_gv_self<<<nblk(nt * 32, 128), 128, 0, s>>>(nt, nrhs, h->k, h->cent, h->qpt, h->nrm, h->area, h->hmax, yx, gs, gel,
                                               dk);
  BEM_CUDA(cudaGetLastError());
  k_gv_finish<<<nblk(nt, 128), 128, 0, s>>>(nt, h->cent, h->qpt, h->nrm, h->area, h->hmax, h->tri, gx, gq, ga, gn,
                                            gel, dV);
  BEM_CUDA(cudaGetLastError());
  BEM_CUDA(cudaMemcpyAsync(dvertices, dV, (size_t)nv * 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  BEM_CUDA(cudaFreeAsync(buf, s));
  return BEM_OK;
}
