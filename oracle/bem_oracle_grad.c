/*
 * bem_oracle_grad.c -- plain FP64 CPU oracle for the derivatives of the
 * collocation operators with respect to the vertex positions and k.
 *
 * TEST INFRASTRUCTURE ONLY, like bem_oracle.c: only the tests, the smoke
 * check and the bench's CPU-baseline leg may load it.  It shares no code with
 * the CUDA library (nor with bem_oracle.c: it restates the same rule-defined
 * entries in its own arithmetic).
 *
 * For z = (1/2 I - D) x + S y (Section 2.3) and a real loss L whose upstream
 * gradient is g = dL/dRe z + i dL/dIm z (PyTorch's convention for complex
 * outputs), dL = sum_rhs sum_i Re(conj(g_i) dz_i), so for any parameter t
 *
 *     dL/dt = sum_rhs sum_{i,j} Re( conj(g_i) (dS_ij/dt y_j - dD_ij/dt x_j) ).
 *
 * The 1/2 I term does not depend on the geometry.  Every entry is recomputed
 * here in forward-mode dual arithmetic (a value and 13 complex tangents): the
 * three coordinates of the collocation point x_i, the nine vertex coordinates
 * of the source triangle Gamma_j, and k.  The rule that defines the entries is
 * the one stated in bem_oracle.c:
 *   - R_0: barycentric (2/3,1/6,1/6) and permutations, weight A/3, on the
 *     triangle or on each of its 4^L midpoint sub-triangles (rule R_L), with
 *     L = 2 / 1 / 0 for |x_i - c_j| < 2 h_j / < 4 h_j / otherwise.  L is
 *     piecewise constant in the vertices, so it carries no derivative.
 *   - i == j: D_ii = 0 for every vertex position (x_i lies in the plane of
 *     Gamma_i), and S_ii is the exact integral: the edge-logarithm closed form
 *     of int 1/r dA plus the polar-coordinate remainder int (exp(ikr)-1)/r dA
 *     with adaptive Gauss-Legendre in the angle.  The panels' end points are
 *     functions of the vertices and carry tangents; panels are halved until
 *     the value and every tangent of the two halves agree with the whole
 *     (tolerances at dclose).
 * x_i is the centroid, so a tangent of x_i moves each vertex of Gamma_i by 1/3.
 * The derivative with respect to k requires k > 0.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define GR_FLAG_RULE1 1
#define GR_FLAG_NO_REFINE 2
#define GR_ND 13 /* tangents: x_i (0..2), source vertices (3..11, vertex-major), k (12) */
#define GR_TK 12

static const double GR_PI = 3.14159265358979323846264338327950288;

/* ---- dual numbers: value + GR_ND complex tangents ---------------------- */
typedef struct {
  cplx v;
  cplx d[GR_ND];
} dual;

static dual dc(cplx v) {
  dual r;
  r.v = v;
  for (int t = 0; t < GR_ND; ++t) r.d[t] = 0.0;
  return r;
}
static dual dvar(double v, int t) {
  dual r = dc(v);
  r.d[t] = 1.0;
  return r;
}
static dual dadd(dual a, dual b) {
  for (int t = 0; t < GR_ND; ++t) a.d[t] += b.d[t];
  a.v += b.v;
  return a;
}
static dual dsub(dual a, dual b) {
  for (int t = 0; t < GR_ND; ++t) a.d[t] -= b.d[t];
  a.v -= b.v;
  return a;
}
static dual dscale(dual a, cplx s) {
  for (int t = 0; t < GR_ND; ++t) a.d[t] *= s;
  a.v *= s;
  return a;
}
static dual dmul(dual a, dual b) {
  dual r;
  r.v = a.v * b.v;
  for (int t = 0; t < GR_ND; ++t) r.d[t] = a.d[t] * b.v + a.v * b.d[t];
  return r;
}
static dual ddiv(dual a, dual b) {
  dual r;
  r.v = a.v / b.v;
  for (int t = 0; t < GR_ND; ++t) r.d[t] = (a.d[t] - r.v * b.d[t]) / b.v;
  return r;
}
/* f(a) with f'(a.v) = fp */
static dual dchain(dual a, cplx f, cplx fp) {
  dual r;
  r.v = f;
  for (int t = 0; t < GR_ND; ++t) r.d[t] = fp * a.d[t];
  return r;
}
static dual dsqrt(dual a) {
  cplx s = csqrt(a.v);
  return dchain(a, s, 0.5 / s);
}
static dual dexp(dual a) {
  cplx e = cexp(a.v);
  return dchain(a, e, e);
}
static dual dlog(dual a) { return dchain(a, clog(a.v), 1.0 / a.v); }
static dual dsin(dual a) { return dchain(a, csin(a.v), ccos(a.v)); }
static dual dcos(dual a) { return dchain(a, ccos(a.v), -csin(a.v)); }
/* atan2 of real-valued duals */
static dual datan2(dual y, dual x) {
  double yv = creal(y.v), xv = creal(x.v), q = xv * xv + yv * yv;
  dual r;
  r.v = atan2(yv, xv);
  for (int t = 0; t < GR_ND; ++t) r.d[t] = (xv * y.d[t] - yv * x.d[t]) / q;
  return r;
}

/* 3-vectors of duals */
static void vsub(const dual* a, const dual* b, dual* o) {
  for (int d = 0; d < 3; ++d) o[d] = dsub(a[d], b[d]);
}
static dual vdot(const dual* a, const dual* b) {
  return dadd(dadd(dmul(a[0], b[0]), dmul(a[1], b[1])), dmul(a[2], b[2]));
}
static void vcross(const dual* a, const dual* b, dual* o) {
  o[0] = dsub(dmul(a[1], b[2]), dmul(a[2], b[1]));
  o[1] = dsub(dmul(a[2], b[0]), dmul(a[0], b[2]));
  o[2] = dsub(dmul(a[0], b[1]), dmul(a[1], b[0]));
}
static dual vnorm(const dual* a) { return dsqrt(vdot(a, a)); }

/* ---- geometry by value (for the rule level) ---------------------------- */
static void tri_values(const double* V, const int32_t* T, int64_t j, double v[3][3], double c[3], double* h) {
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) v[a][d] = V[3 * (int64_t)T[3 * j + a] + d];
  double hm = 0.0;
  for (int a = 0; a < 3; ++a) {
    double e2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      double e = v[(a + 1) % 3][d] - v[a][d];
      e2 += e * e;
    }
    hm = fmax(hm, sqrt(e2));
  }
  for (int d = 0; d < 3; ++d) c[d] = (v[0][d] + v[1][d] + v[2][d]) / 3.0;
  *h = hm;
}

/* ---- the kernels at one point ------------------------------------------ */
/* s += w G(x - y), dd += w dG/dn_y; G = exp(ikr)/(4 pi r) */
static void dkernel_add(const dual* x, const dual* y, const dual* n, dual w, dual k, dual* s, dual* dd) {
  dual r3[3];
  vsub(y, x, r3);
  dual r = vnorm(r3);
  dual ikr = dscale(dmul(k, r), I);
  dual e = dexp(ikr);
  dual g = ddiv(e, dscale(r, 4.0 * GR_PI));
  *s = dadd(*s, dmul(w, g));
  dual r3c = dmul(dmul(r, r), r);
  dual f = ddiv(dmul(e, dsub(ikr, dc(1.0))), dscale(r3c, 4.0 * GR_PI));
  *dd = dadd(*dd, dmul(w, dmul(f, vdot(r3, n))));
}

/* rule R_L on the triangle (a, b, c) with normal n */
static void drule(const dual* x, const dual* a, const dual* b, const dual* c, const dual* n, int L, dual k, dual* s,
                  dual* dd) {
  if (L == 0) {
    dual e1[3], e2[3], cr[3];
    vsub(b, a, e1);
    vsub(c, a, e2);
    vcross(e1, e2, cr);
    dual w = dscale(vnorm(cr), 0.5 / 3.0);
    const double bary[3][3] = {{2.0 / 3, 1.0 / 6, 1.0 / 6}, {1.0 / 6, 2.0 / 3, 1.0 / 6}, {1.0 / 6, 1.0 / 6, 2.0 / 3}};
    for (int q = 0; q < 3; ++q) {
      dual y[3];
      for (int d = 0; d < 3; ++d)
        y[d] = dadd(dadd(dscale(a[d], bary[q][0]), dscale(b[d], bary[q][1])), dscale(c[d], bary[q][2]));
      dkernel_add(x, y, n, w, k, s, dd);
    }
    return;
  }
  dual ab[3], bc[3], ca[3];
  for (int d = 0; d < 3; ++d) {
    ab[d] = dscale(dadd(a[d], b[d]), 0.5);
    bc[d] = dscale(dadd(b[d], c[d]), 0.5);
    ca[d] = dscale(dadd(c[d], a[d]), 0.5);
  }
  drule(x, a, ab, ca, n, L - 1, k, s, dd);
  drule(x, ab, b, bc, n, L - 1, k, s, dd);
  drule(x, ca, bc, c, n, L - 1, k, s, dd);
  drule(x, ab, bc, ca, n, L - 1, k, s, dd);
}

/* unit normal (b - a) x (c - a) / |.| */
static void dnormal(const dual v[3][3], dual* n) {
  dual e1[3], e2[3], cr[3];
  vsub(v[1], v[0], e1);
  vsub(v[2], v[0], e2);
  vcross(e1, e2, cr);
  dual len = vnorm(cr);
  for (int d = 0; d < 3; ++d) n[d] = ddiv(cr[d], len);
}

/* ---- exact self term in dual arithmetic ---------------------------------- */
#define GR_GL_N 16
static double gr_x[GR_GL_N], gr_w[GR_GL_N];
static int gr_ready = 0;

static void gr_gl_init(void) {
  if (gr_ready) return;
  int n = GR_GL_N;
  for (int i = 0; i < n; ++i) {
    double z = cos(GR_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int m = 2; m <= n; ++m) {
        double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int m = 2; m <= n; ++m) {
      double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    gr_x[i] = z;
    gr_w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  gr_ready = 1;
}

/* radial integral of (exp(ikr) - 1)/r * r dr from 0 to rho = dist / cos(phi):
 * (exp(ik rho) - 1)/(ik) - rho = sin(k rho)/k - rho + i (1 - cos(k rho))/k */
static dual dsmooth_radial(dual dist, dual phi, dual k) {
  dual rho = ddiv(dist, dcos(phi));
  dual kr = dmul(k, rho);
  dual sh = dsin(dscale(kr, 0.5));
  dual re = dsub(ddiv(dsin(kr), k), rho);
  dual im = ddiv(dscale(dmul(sh, sh), 2.0), k);
  return dadd(re, dscale(im, I));
}

static dual dgl_panel(dual dist, dual a, dual b, dual k) {
  dual half = dscale(dsub(b, a), 0.5), mid = dscale(dadd(a, b), 0.5);
  dual s = dc(0.0);
  for (int q = 0; q < GR_GL_N; ++q) {
    dual phi = dadd(mid, dscale(half, gr_x[q]));
    s = dadd(s, dscale(dsmooth_radial(dist, phi, k), gr_w[q]));
  }
  return dmul(half, s);
}

/* A panel is accepted when its halves agree with it: the value to the tolerance
 * bem_oracle.c uses, each tangent to 1e-13 of the whole edge integral's
 * tangent (floored at 1) per unit of angle.  A budget of panels per edge bounds
 * the recursion where rounding keeps the tangents from settling. */
static int dclose(dual lr, dual whole, const dual* top, double width) {
  if (cabs(lr.v - whole.v) > 1e-15 * (1.0 + cabs(lr.v)) * width) return 0;
  for (int t = 0; t < GR_ND; ++t)
    if (cabs(lr.d[t] - whole.d[t]) > 1e-13 * (1.0 + cabs(top->d[t])) * width) return 0;
  return 1;
}

static dual dgl_adaptive(dual dist, dual a, dual b, dual k, dual whole, const dual* top, int depth, int* budget) {
  dual m = dscale(dadd(a, b), 0.5);
  dual l = dgl_panel(dist, a, m, k), r = dgl_panel(dist, m, b, k);
  dual lr = dadd(l, r);
  *budget -= 2;
  if (depth >= 40 || *budget <= 0 || dclose(lr, whole, top, creal(b.v) - creal(a.v))) return lr;
  dual left = dgl_adaptive(dist, a, m, k, l, top, depth + 1, budget);
  return dadd(left, dgl_adaptive(dist, m, b, k, r, top, depth + 1, budget));
}

/* S_ii of the triangle v at its own centroid */
static dual dself(const dual v[3][3], dual k) {
  dual x[3];
  for (int d = 0; d < 3; ++d) x[d] = dscale(dadd(dadd(v[0][d], v[1][d]), v[2][d]), 1.0 / 3.0);
  dual s_static = dc(0.0), s_smooth = dc(0.0);
  for (int e = 0; e < 3; ++e) {
    const dual* a = v[e];
    const dual* b = v[(e + 1) % 3];
    dual ab[3], xa[3], tv[3], foot[3], xf[3], bf[3], af[3], bx[3];
    vsub(b, a, ab);
    dual len = vnorm(ab);
    for (int d = 0; d < 3; ++d) tv[d] = ddiv(ab[d], len);
    vsub(x, a, xa);
    dual proj = vdot(xa, tv);
    for (int d = 0; d < 3; ++d) foot[d] = dadd(a[d], dmul(proj, tv[d]));
    vsub(x, foot, xf);
    dual dist = vnorm(xf);
    vsub(b, foot, bf);
    vsub(a, foot, af);
    dual sp = vdot(bf, tv), sm = vdot(af, tv);
    vsub(b, x, bx);
    dual Rp = vnorm(bx), Rm = vnorm(xa);
    s_static = dadd(s_static, dmul(dist, dlog(ddiv(dadd(Rp, sp), dadd(Rm, sm)))));
    dual phip = datan2(sp, dist), phim = datan2(sm, dist);
    dual top = dgl_panel(dist, phim, phip, k);
    int budget = 1 << 22;
    s_smooth = dadd(s_smooth, dgl_adaptive(dist, phim, phip, k, top, &top, 0, &budget));
  }
  return dscale(dadd(s_static, s_smooth), 1.0 / (4.0 * GR_PI));
}

/* ---- one pair ------------------------------------------------------------ */
/* dS, dD of entry (i, j).  Tangents: x_i 0..2 (unused when i == j), vertices of
 * Gamma_j 3..11, k 12. */
static void dentry(const double* V, const int32_t* T, int64_t i, int64_t j, double k, int flags, dual* s,
                   dual* dd) {
  double vi[3][3], ci[3], hi, vj[3][3], cj[3], hj;
  tri_values(V, T, i, vi, ci, &hi);
  tri_values(V, T, j, vj, cj, &hj);
  dual kk = dvar(k, GR_TK);
  dual v[3][3];
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) v[a][d] = dvar(vj[a][d], 3 + 3 * a + d);
  *s = dc(0.0);
  *dd = dc(0.0);
  if (i == j) {
    *s = dself(v, kk);
    return;
  }
  dual x[3];
  for (int d = 0; d < 3; ++d) x[d] = dvar(ci[d], d);
  dual n[3];
  dnormal(v, n);
  if (flags & GR_FLAG_RULE1) {
    dual e1[3], e2[3], cr[3], c[3];
    vsub(v[1], v[0], e1);
    vsub(v[2], v[0], e2);
    vcross(e1, e2, cr);
    for (int d = 0; d < 3; ++d) c[d] = dscale(dadd(dadd(v[0][d], v[1][d]), v[2][d]), 1.0 / 3.0);
    dkernel_add(x, c, n, dscale(vnorm(cr), 0.5), kk, s, dd);
    return;
  }
  int L = 0;
  if (!(flags & GR_FLAG_NO_REFINE)) {
    double dx = ci[0] - cj[0], dy = ci[1] - cj[1], dz = ci[2] - cj[2];
    double dist = sqrt(dx * dx + dy * dy + dz * dz);
    L = dist < 2.0 * hj ? 2 : (dist < 4.0 * hj ? 1 : 0);
  }
  drule(x, v[0], v[1], v[2], n, L, kk, s, dd);
}

/* adds the pair's contribution to the vertex gradient and dk */
static void accumulate(const int32_t* T, int64_t nt, int nrhs, int64_t i, int64_t j, const dual* s, const dual* dd,
                       const cplx* g, const cplx* x, const cplx* y, double* dV, double* dk) {
  cplx cs = 0.0, cd = 0.0;
  for (int r = 0; r < nrhs; ++r) {
    cplx gi = conj(g[(int64_t)r * nt + i]);
    if (y) cs += gi * y[(int64_t)r * nt + j];
    if (x) cd += gi * x[(int64_t)r * nt + j];
  }
  double val[GR_ND];
  for (int t = 0; t < GR_ND; ++t) val[t] = creal(cs * s->d[t] - cd * dd->d[t]);
  if (i != j)
    for (int a = 0; a < 3; ++a)
      for (int d = 0; d < 3; ++d) dV[3 * (int64_t)T[3 * i + a] + d] += val[d] / 3.0;
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) dV[3 * (int64_t)T[3 * j + a] + d] += val[3 + 3 * a + d];
  *dk += val[GR_TK];
}

/*
 * Gradient of L (see the file header) with respect to the vertices and k.
 *   g, x, y : interleaved complex [nrhs][nt]; x or y may be NULL (treated as 0).
 *   vsel    : NULL -> every pair; dV is [nv][3] and dk (nullable) is filled.
 *             otherwise only the pairs that involve a triangle touching one of
 *             the nvsel listed vertices; dV is [nvsel][3] in the listed order
 *             and dk must be NULL.
 * Returns 0, or 1 on bad arguments / allocation failure.
 */
int oracle_grad(const double* V, int64_t nv, const int32_t* T, int64_t nt, double k, int flags, int nrhs,
                const double* g, const double* x, const double* y, const int64_t* vsel, int64_t nvsel, double* dV,
                double* dk) {
  if (!g || (!x && !y) || k <= 0.0 || (vsel && dk)) return 1;
  gr_gl_init();
  const cplx* gc = (const cplx*)g;
  const cplx* xc = (const cplx*)x;
  const cplx* yc = (const cplx*)y;
  char* mark = (char*)calloc((size_t)nt, 1);
  int64_t* marked = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nt > 0 ? nt : 1));
  if (!mark || !marked) {
    free(mark);
    free(marked);
    return 1;
  }
  int64_t nmarked = 0;
  if (vsel) {
    char* vm = (char*)calloc((size_t)nv, 1);
    if (!vm) {
      free(mark);
      free(marked);
      return 1;
    }
    for (int64_t s = 0; s < nvsel; ++s) vm[vsel[s]] = 1;
    for (int64_t j = 0; j < nt; ++j)
      if (vm[T[3 * j]] || vm[T[3 * j + 1]] || vm[T[3 * j + 2]]) {
        mark[j] = 1;
        marked[nmarked++] = j;
      }
    free(vm);
  }
  double* total = (double*)calloc((size_t)(3 * nv), sizeof(double));
  double dk_total = 0.0;
  int failed = total == NULL;
#pragma omp parallel reduction(+ : dk_total)
  {
    double* acc = (double*)calloc((size_t)(3 * nv), sizeof(double));
    double dk_part = 0.0;
    if (!acc) {
#pragma omp atomic write
      failed = 1;
    }
#pragma omp for schedule(dynamic, 8)
    for (int64_t i = 0; i < nt; ++i) {
      if (!acc) continue;
      int all = !vsel || mark[i];
      int64_t cnt = all ? nt : nmarked;
      for (int64_t q = 0; q < cnt; ++q) {
        int64_t j = all ? q : marked[q];
        dual s, dd;
        dentry(V, T, i, j, k, flags, &s, &dd);
        accumulate(T, nt, nrhs, i, j, &s, &dd, gc, xc, yc, acc, &dk_part);
      }
    }
    if (acc && total) {
#pragma omp critical
      for (int64_t e = 0; e < 3 * nv; ++e) total[e] += acc[e];
    }
    free(acc);
    dk_total += dk_part;
  }
  if (!failed) {
    if (vsel) {
      for (int64_t s = 0; s < nvsel; ++s)
        for (int d = 0; d < 3; ++d) dV[3 * s + d] = total[3 * vsel[s] + d];
    } else {
      memcpy(dV, total, sizeof(double) * (size_t)(3 * nv));
      if (dk) *dk = dk_total;
    }
  }
  free(total);
  free(mark);
  free(marked);
  return failed;
}
