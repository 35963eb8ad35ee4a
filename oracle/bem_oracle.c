/*
 * bem_oracle.c -- plain FP64 CPU oracle for the collocation BEM operators.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg may load this library; the product path never does.  It
 * shares no code, header or table with the CUDA library.
 *
 * What it computes (Section 2.3 of the paper, Eq. (danseibie2) and the block
 * system Eq. (renritupu)): for a surface made of flat triangles Gamma_j with
 * piecewise-constant densities and collocation at the centroids x_i,
 *
 *     z = (1/2 I - D) x + S y,
 *     S_ij = int_{Gamma_j} G(x_i - y) dGamma_y,
 *     D_ij = int_{Gamma_j} dG/dn_y (x_i - y) dGamma_y,
 *     G(r) = exp(i k r) / (4 pi r)                      (Section 2.3),
 *     dG/dn_y = exp(i k r)(i k r - 1)/(4 pi r^3) (y - x).n_j,
 *
 * with n_j the unit normal pointing out of the scatterer into the fluid
 * (Section 2.1).  The paper fixes no quadrature, so the rule that *defines*
 * each matrix entry is stated here and written out plainly:
 *
 *   R_0   3-point symmetric rule: barycentric (2/3,1/6,1/6) and permutations,
 *         each weight A_j/3.
 *   R_L   the triangle split uniformly L times (4^L congruent pieces, edge
 *         midpoints) with R_0 on every piece.
 *   i!=j  L = 2 if |x_i - c_j| < 2 h_j, L = 1 if < 4 h_j, else L = 0
 *         (c_j centroid, h_j longest edge).
 *   i==j  D_ii = 0 (flat element: (y - x_i).n_i = 0); S_ii is the exact
 *         integral: the closed-form potential of a uniform flat triangle at an
 *         interior point, int 1/r dA = sum_edges d ln((R+ + s+)/(R- + s-)),
 *         plus the bounded remainder int (exp(ikr)-1)/r dA done in polar
 *         coordinates about x_i, where the radial integral is analytic and the
 *         angle integral is adaptive Gauss-Legendre (16-point panels halved
 *         until the halves agree to 1e-15) per edge.
 *
 * A 1-point (centroid) rule without near refinement is available through
 * flags; it exists for the reciprocity pin (S_ij/A_j = S_ji/A_i exactly).
 *
 * Dense solves use an unblocked right-looking LU with partial pivoting (the
 * role LAPACK ZGESV plays in Section 3.1).
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

#define OR_FLAG_RULE1 1     /* 1-point centroid rule for regular entries      */
#define OR_FLAG_NO_REFINE 2 /* no near-singular subdivision (R_0 everywhere)  */
#define OR_FLAG_NO_HALF 4   /* omit the 1/2 I term                            */

static const double OR_PI = 3.14159265358979323846264338327950288;

typedef struct {
  double v[3][3]; /* vertices */
  double c[3];    /* centroid */
  double n[3];    /* unit normal */
  double area;
  double h;       /* longest edge */
} tri_t;

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double* a) { return sqrt(dot3(a, a)); }
static void sub3(const double* a, const double* b, double* o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static void cross3(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

static void tri_load(const double* V, const int32_t* T, int64_t j, tri_t* t) {
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) t->v[a][d] = V[3 * (int64_t)T[3 * j + a] + d];
  double e1[3], e2[3], e3[3], cr[3];
  sub3(t->v[1], t->v[0], e1);
  sub3(t->v[2], t->v[0], e2);
  sub3(t->v[2], t->v[1], e3);
  cross3(e1, e2, cr);
  double len = norm3(cr);
  t->area = 0.5 * len;
  for (int d = 0; d < 3; ++d) {
    t->n[d] = cr[d] / len;
    t->c[d] = (t->v[0][d] + t->v[1][d] + t->v[2][d]) / 3.0;
  }
  double h1 = norm3(e1), h2 = norm3(e2), h3 = norm3(e3);
  t->h = fmax(h1, fmax(h2, h3));
}

/* ---- kernels ---------------------------------------------------------- */

/* add w*G(x-y) to *s and w*dG/dn_y to *d */
static void kernel_add(const double* x, const double* y, const double* n, double w, double k, cplx* s, cplx* d) {
  double r3[3];
  sub3(y, x, r3); /* y - x */
  double r = norm3(r3);
  cplx e = cexp(I * k * r);
  cplx g = e / (4.0 * OR_PI * r);
  *s += w * g;
  *d += w * e * (I * k * r - 1.0) / (4.0 * OR_PI * r * r * r) * dot3(r3, n);
}

/* rule R_L on the triangle (a,b,c) with normal n */
static void rule_rl(const double* x, const double* a, const double* b, const double* c, const double* n, int L,
                    double k, cplx* s, cplx* d) {
  if (L == 0) {
    double e1[3], e2[3], cr[3];
    sub3(b, a, e1);
    sub3(c, a, e2);
    cross3(e1, e2, cr);
    double w = 0.5 * norm3(cr) / 3.0;
    double bary[3][3] = {{2.0 / 3, 1.0 / 6, 1.0 / 6}, {1.0 / 6, 2.0 / 3, 1.0 / 6}, {1.0 / 6, 1.0 / 6, 2.0 / 3}};
    for (int q = 0; q < 3; ++q) {
      double y[3];
      for (int dd = 0; dd < 3; ++dd) y[dd] = bary[q][0] * a[dd] + bary[q][1] * b[dd] + bary[q][2] * c[dd];
      kernel_add(x, y, n, w, k, s, d);
    }
    return;
  }
  double ab[3], bc[3], ca[3];
  for (int dd = 0; dd < 3; ++dd) {
    ab[dd] = 0.5 * (a[dd] + b[dd]);
    bc[dd] = 0.5 * (b[dd] + c[dd]);
    ca[dd] = 0.5 * (c[dd] + a[dd]);
  }
  rule_rl(x, a, ab, ca, n, L - 1, k, s, d);
  rule_rl(x, ab, b, bc, n, L - 1, k, s, d);
  rule_rl(x, ca, bc, c, n, L - 1, k, s, d);
  rule_rl(x, ab, bc, ca, n, L - 1, k, s, d);
}

/* ---- Gauss-Legendre nodes (Newton iteration on P_n) --------------------- */
#define OR_GL_N 16
static double gl_x[OR_GL_N], gl_w[OR_GL_N];
static int gl_ready = 0;

static void gl_init(void) {
  if (gl_ready) return;
  int n = OR_GL_N;
  for (int i = 0; i < n; ++i) {
    double z = cos(OR_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
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
    gl_x[i] = z;
    gl_w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  gl_ready = 1;
}

/* ---- exact self term S_ii --------------------------------------------- */
/* Remainder integrand in polar coordinates about the centroid, for the edge
 * at distance `dist`: the radial integral of (exp(ikr)-1)/r r dr from 0 to
 * rho = dist / cos(phi) is (exp(ik rho)-1)/(ik) - rho. */
static cplx smooth_radial(double dist, double phi, double k) {
  double rho = dist / cos(phi);
  if (k == 0.0) return 0.0;
  double sh = sin(0.5 * k * rho);
  return (sin(k * rho) / k - rho) + I * (2.0 * sh * sh / k);
}

static cplx gl_panel(double dist, double a, double b, double k) {
  double half = 0.5 * (b - a), mid = 0.5 * (a + b);
  cplx s = 0.0;
  for (int q = 0; q < OR_GL_N; ++q) s += gl_w[q] * smooth_radial(dist, mid + half * gl_x[q], k);
  return half * s;
}

/* adaptive: bisect a panel until its two halves agree with it */
static cplx gl_adaptive(double dist, double a, double b, double k, cplx whole, int depth) {
  double m = 0.5 * (a + b);
  cplx l = gl_panel(dist, a, m, k), r = gl_panel(dist, m, b, k);
  if (depth >= 40 || cabs(l + r - whole) <= 1e-15 * (1.0 + cabs(l + r)) * (b - a)) return l + r;
  return gl_adaptive(dist, a, m, k, l, depth + 1) + gl_adaptive(dist, m, b, k, r, depth + 1);
}

/* Returns S_ii for the triangle t at its own centroid.  See file header. */
static cplx self_single_layer(const tri_t* t, double k) {
  const double* x = t->c;
  double s_static = 0.0;  /* int 1/r dA */
  cplx s_smooth = 0.0;    /* int (exp(ikr)-1)/r dA */
  for (int e = 0; e < 3; ++e) {
    const double* a = t->v[e];
    const double* b = t->v[(e + 1) % 3];
    double ab[3], xa[3];
    sub3(b, a, ab);
    double len = norm3(ab);
    double tv[3] = {ab[0] / len, ab[1] / len, ab[2] / len};
    sub3(x, a, xa);
    double proj = dot3(xa, tv);
    double foot[3] = {a[0] + proj * tv[0], a[1] + proj * tv[1], a[2] + proj * tv[2]};
    double xf[3], bf[3], af[3], bx[3];
    sub3(x, foot, xf);
    double dist = norm3(xf);
    sub3(b, foot, bf);
    sub3(a, foot, af);
    double sp = dot3(bf, tv), sm = dot3(af, tv);
    sub3(b, x, bx);
    double Rp = norm3(bx), Rm = norm3(xa);
    s_static += dist * log((Rp + sp) / (Rm + sm));
    double phip = atan2(sp, dist), phim = atan2(sm, dist);
    s_smooth += gl_adaptive(dist, phim, phip, k, gl_panel(dist, phim, phip, k), 0);
  }
  return (s_static + s_smooth) / (4.0 * OR_PI);
}

/* ---- one matrix entry --------------------------------------------------- */
static int choose_level(const double* x, const tri_t* tj, int flags) {
  if (flags & (OR_FLAG_NO_REFINE | OR_FLAG_RULE1)) return 0;
  double dx[3];
  sub3(x, tj->c, dx);
  double dist = norm3(dx);
  if (dist < 2.0 * tj->h) return 2;
  if (dist < 4.0 * tj->h) return 1;
  return 0;
}

/* S and D entries for target point x against triangle j (x not on Gamma_j) */
static void entry_offsurface(const double* x, const tri_t* tj, double k, int flags, cplx* s, cplx* d) {
  *s = 0.0;
  *d = 0.0;
  if (flags & OR_FLAG_RULE1) {
    kernel_add(x, tj->c, tj->n, tj->area, k, s, d);
    return;
  }
  int L = choose_level(x, tj, flags);
  rule_rl(x, tj->v[0], tj->v[1], tj->v[2], tj->n, L, k, s, d);
}

static void entry(const tri_t* ti, int64_t i, const tri_t* tj, int64_t j, double k, int flags, cplx* s, cplx* d) {
  if (i == j) {
    *s = self_single_layer(ti, k);
    *d = 0.0;
    return;
  }
  entry_offsurface(ti->c, tj, k, flags, s, d);
}

/* ---- gradient of the entries with respect to the field point ------------
   With d = y - x, r = |d|, F = exp(ikr)(ikr - 1)/(4 pi r^3) and
   H = exp(ikr)(3 - 3ikr - k^2 r^2)/(4 pi r^5) (dF/dr = -r H):
     grad_x G          = -F d
     grad_x dG/dn_y    = -(H (d.n) d + F n)
   from G = exp(ikr)/(4 pi r) and dG/dn_y = F (d.n). */
static void kernel_grad_add(const double* x, const double* y, const double* n, double w, double k, cplx gs[3],
                            cplx gd[3]) {
  double dv[3];
  sub3(y, x, dv);
  double r = norm3(dv);
  cplx e = cexp(I * k * r);
  cplx F = e * (I * k * r - 1.0) / (4.0 * OR_PI * r * r * r);
  cplx H = e * (3.0 - 3.0 * I * k * r - k * k * r * r) / (4.0 * OR_PI * r * r * r * r * r);
  double dn = dot3(dv, n);
  for (int c = 0; c < 3; ++c) {
    gs[c] += -w * F * dv[c];
    gd[c] += -w * (H * dn * dv[c] + F * n[c]);
  }
}

/* the gradient entries under the rule R_L (same pieces and points as rule_rl) */
static void rule_rl_grad(const double* x, const double* a, const double* b, const double* c, const double* n, int L,
                         double k, cplx gs[3], cplx gd[3]) {
  if (L == 0) {
    double e1[3], e2[3], cr[3];
    sub3(b, a, e1);
    sub3(c, a, e2);
    cross3(e1, e2, cr);
    double w = 0.5 * norm3(cr) / 3.0;
    double bary[3][3] = {{2.0 / 3, 1.0 / 6, 1.0 / 6}, {1.0 / 6, 2.0 / 3, 1.0 / 6}, {1.0 / 6, 1.0 / 6, 2.0 / 3}};
    for (int q = 0; q < 3; ++q) {
      double y[3];
      for (int dd = 0; dd < 3; ++dd) y[dd] = bary[q][0] * a[dd] + bary[q][1] * b[dd] + bary[q][2] * c[dd];
      kernel_grad_add(x, y, n, w, k, gs, gd);
    }
    return;
  }
  double ab[3], bc[3], ca[3];
  for (int dd = 0; dd < 3; ++dd) {
    ab[dd] = 0.5 * (a[dd] + b[dd]);
    bc[dd] = 0.5 * (b[dd] + c[dd]);
    ca[dd] = 0.5 * (c[dd] + a[dd]);
  }
  rule_rl_grad(x, a, ab, ca, n, L - 1, k, gs, gd);
  rule_rl_grad(x, ab, b, bc, n, L - 1, k, gs, gd);
  rule_rl_grad(x, ca, bc, c, n, L - 1, k, gs, gd);
  rule_rl_grad(x, ab, bc, ca, n, L - 1, k, gs, gd);
}

/* ---- public API --------------------------------------------------------- */

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Per-triangle geometry: centroid[3nt], area[nt], normal[3nt], hmax[nt]. */
int oracle_geometry(const double* V, int64_t nv, const int32_t* T, int64_t nt, double* cent, double* area,
                    double* normal, double* hmax) {
  (void)nv;
  for (int64_t j = 0; j < nt; ++j) {
    tri_t t;
    tri_load(V, T, j, &t);
    for (int d = 0; d < 3; ++d) {
      if (cent) cent[3 * j + d] = t.c[d];
      if (normal) normal[3 * j + d] = t.n[d];
    }
    if (area) area[j] = t.area;
    if (hmax) hmax[j] = t.h;
  }
  return 0;
}

/* Single entries S_ij, D_ij for a list of (i,j) pairs. out: interleaved complex [npairs][2] (S then D). */
int oracle_entries(const double* V, int64_t nv, const int32_t* T, int64_t nt, double k, int flags,
                   const int64_t* ii, const int64_t* jj, int64_t npairs, double* out) {
  (void)nv;
  (void)nt;
  gl_init();
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t p = 0; p < npairs; ++p) {
    tri_t ti, tj;
    tri_load(V, T, ii[p], &ti);
    tri_load(V, T, jj[p], &tj);
    cplx s, d;
    entry(&ti, ii[p], &tj, jj[p], k, flags, &s, &d);
    out[4 * p + 0] = creal(s);
    out[4 * p + 1] = cimag(s);
    out[4 * p + 2] = creal(d);
    out[4 * p + 3] = cimag(d);
  }
  return 0;
}

/*
 * z[r][row] = 1/2 x[r][i] - sum_j D_ij x[r][j] + sum_j S_ij y[r][j] for i = rows[row]
 * (all rows when rows == NULL, nrows ignored).  x, y nullable (treated as 0).
 * Complex arrays are interleaved (re, im), layout [nrhs][nt] (z: [nrhs][nrows]).
 */
int oracle_apply(const double* V, int64_t nv, const int32_t* T, int64_t nt, double k, int flags, int nrhs,
                 const double* x, const double* y, double* z, const int64_t* rows, int64_t nrows) {
  (void)nv;
  gl_init();
  if (!rows) nrows = nt;
  tri_t* tris = (tri_t*)malloc(sizeof(tri_t) * (size_t)nt);
  if (!tris) return 1;
  for (int64_t j = 0; j < nt; ++j) tri_load(V, T, j, &tris[j]);
  const cplx* xc = (const cplx*)x;
  const cplx* yc = (const cplx*)y;
  cplx* zc = (cplx*)z;
#pragma omp parallel
  {
    cplx* acc = (cplx*)malloc(sizeof(cplx) * (size_t)nrhs);
#pragma omp for schedule(dynamic, 1)
    for (int64_t r = 0; r < nrows; ++r) {
      int64_t i = rows ? rows[r] : r;
      for (int q = 0; q < nrhs; ++q) acc[q] = 0.0;
      for (int64_t j = 0; j < nt; ++j) {
        cplx s, d;
        entry(&tris[i], i, &tris[j], j, k, flags, &s, &d);
        for (int q = 0; q < nrhs; ++q) {
          if (yc) acc[q] += s * yc[(int64_t)q * nt + j];
          if (xc) acc[q] -= d * xc[(int64_t)q * nt + j];
        }
      }
      for (int q = 0; q < nrhs; ++q) {
        cplx half = (xc && !(flags & OR_FLAG_NO_HALF)) ? 0.5 * xc[(int64_t)q * nt + i] : 0.0;
        zc[(int64_t)q * nrows + r] = half + acc[q];
      }
    }
    free(acc);
  }
  free(tris);
  return 0;
}

/*
 * Conjugate-transpose apply: gx = (1/2 I - D)^H g, gy = S^H g (either nullable).
 * gx[j] = 1/2 g[j] - sum_i conj(D_ij) g[i];  gy[j] = sum_i conj(S_ij) g[i].
 */
int oracle_apply_adjoint(const double* V, int64_t nv, const int32_t* T, int64_t nt, double k, int flags, int nrhs,
                         const double* g, double* gx, double* gy) {
  (void)nv;
  gl_init();
  tri_t* tris = (tri_t*)malloc(sizeof(tri_t) * (size_t)nt);
  if (!tris) return 1;
  for (int64_t j = 0; j < nt; ++j) tri_load(V, T, j, &tris[j]);
  const cplx* gc = (const cplx*)g;
  cplx* gxc = (cplx*)gx;
  cplx* gyc = (cplx*)gy;
#pragma omp parallel
  {
    cplx* ax = (cplx*)malloc(sizeof(cplx) * (size_t)nrhs);
    cplx* ay = (cplx*)malloc(sizeof(cplx) * (size_t)nrhs);
#pragma omp for schedule(dynamic, 1)
    for (int64_t j = 0; j < nt; ++j) {
      for (int q = 0; q < nrhs; ++q) ax[q] = ay[q] = 0.0;
      for (int64_t i = 0; i < nt; ++i) {
        cplx s, d;
        entry(&tris[i], i, &tris[j], j, k, flags, &s, &d);
        for (int q = 0; q < nrhs; ++q) {
          cplx gi = gc[(int64_t)q * nt + i];
          ay[q] += conj(s) * gi;
          ax[q] -= conj(d) * gi;
        }
      }
      for (int q = 0; q < nrhs; ++q) {
        cplx half = (flags & OR_FLAG_NO_HALF) ? 0.0 : 0.5 * gc[(int64_t)q * nt + j];
        if (gxc) gxc[(int64_t)q * nt + j] = half + ax[q];
        if (gyc) gyc[(int64_t)q * nt + j] = ay[q];
      }
    }
    free(ax);
    free(ay);
  }
  free(tris);
  return 0;
}

/*
 * Layer potentials at arbitrary points off the surface:
 * out[r][p] = sum_j S(p, j) y[r][j] - D(p, j) x[r][j]   (rule by distance, no self term)
 */
int oracle_eval_points(const double* V, int64_t nv, const int32_t* T, int64_t nt, double k, int flags, int nrhs,
                       const double* x, const double* y, const double* pts, int64_t npts, double* out) {
  (void)nv;
  gl_init();
  tri_t* tris = (tri_t*)malloc(sizeof(tri_t) * (size_t)nt);
  if (!tris) return 1;
  for (int64_t j = 0; j < nt; ++j) tri_load(V, T, j, &tris[j]);
  const cplx* xc = (const cplx*)x;
  const cplx* yc = (const cplx*)y;
  cplx* oc = (cplx*)out;
#pragma omp parallel
  {
    cplx* acc = (cplx*)malloc(sizeof(cplx) * (size_t)nrhs);
#pragma omp for schedule(dynamic, 1)
    for (int64_t p = 0; p < npts; ++p) {
      for (int q = 0; q < nrhs; ++q) acc[q] = 0.0;
      for (int64_t j = 0; j < nt; ++j) {
        cplx s, d;
        entry_offsurface(&pts[3 * p], &tris[j], k, flags, &s, &d);
        for (int q = 0; q < nrhs; ++q) {
          if (yc) acc[q] += s * yc[(int64_t)q * nt + j];
          if (xc) acc[q] -= d * xc[(int64_t)q * nt + j];
        }
      }
      for (int q = 0; q < nrhs; ++q) oc[(int64_t)q * npts + p] = acc[q];
    }
    free(acc);
  }
  free(tris);
  return 0;
}

/* grad u(p) for u(p) = sum_j S(p, j) y_j - D(p, j) x_j (the entries' rules),
   out [nrhs][npts][3] complex */
int oracle_eval_points_grad(const double* V, int64_t nv, const int32_t* T, int64_t nt, double k, int flags,
                            int nrhs, const double* x, const double* y, const double* pts, int64_t npts,
                            double* out) {
  (void)nv;
  tri_t* tris = (tri_t*)malloc(sizeof(tri_t) * (size_t)nt);
  if (!tris) return 1;
  for (int64_t j = 0; j < nt; ++j) tri_load(V, T, j, &tris[j]);
  const cplx* xc = (const cplx*)x;
  const cplx* yc = (const cplx*)y;
  cplx* oc = (cplx*)out;
#pragma omp parallel
  {
    cplx* acc = (cplx*)malloc(sizeof(cplx) * 3 * (size_t)nrhs);
#pragma omp for schedule(dynamic, 1)
    for (int64_t p = 0; p < npts; ++p) {
      for (int q = 0; q < 3 * nrhs; ++q) acc[q] = 0.0;
      for (int64_t j = 0; j < nt; ++j) {
        cplx gs[3] = {0.0, 0.0, 0.0}, gd[3] = {0.0, 0.0, 0.0};
        const tri_t* tj = &tris[j];
        if (flags & OR_FLAG_RULE1) {
          kernel_grad_add(&pts[3 * p], tj->c, tj->n, tj->area, k, gs, gd);
        } else {
          int L = choose_level(&pts[3 * p], tj, flags);
          rule_rl_grad(&pts[3 * p], tj->v[0], tj->v[1], tj->v[2], tj->n, L, k, gs, gd);
        }
        for (int q = 0; q < nrhs; ++q)
          for (int c = 0; c < 3; ++c) {
            if (yc) acc[3 * q + c] += gs[c] * yc[(int64_t)q * nt + j];
            if (xc) acc[3 * q + c] -= gd[c] * xc[(int64_t)q * nt + j];
          }
      }
      for (int q = 0; q < nrhs; ++q)
        for (int c = 0; c < 3; ++c) oc[((int64_t)q * npts + p) * 3 + c] = acc[3 * q + c];
    }
    free(acc);
  }
  free(tris);
  return 0;
}

/* Dense matrices S and D (row-major, interleaved complex [nt][nt]); either nullable. */
int oracle_assemble(const double* V, int64_t nv, const int32_t* T, int64_t nt, double k, int flags, double* Smat,
                    double* Dmat) {
  (void)nv;
  gl_init();
  tri_t* tris = (tri_t*)malloc(sizeof(tri_t) * (size_t)nt);
  if (!tris) return 1;
  for (int64_t j = 0; j < nt; ++j) tri_load(V, T, j, &tris[j]);
  cplx* S = (cplx*)Smat;
  cplx* D = (cplx*)Dmat;
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t i = 0; i < nt; ++i) {
    for (int64_t j = 0; j < nt; ++j) {
      cplx s, d;
      entry(&tris[i], i, &tris[j], j, k, flags, &s, &d);
      if (S) S[i * nt + j] = s;
      if (D) D[i * nt + j] = d;
    }
  }
  free(tris);
  return 0;
}

/*
 * Solve A X = B in place by LU with partial pivoting.  A: row-major complex
 * [n][n] (overwritten by its factors); B: [nrhs][n] (overwritten by X).
 * Returns 0, or 2 on an exactly singular pivot.
 */
int oracle_lu_solve(int64_t n, double* A_, int nrhs, double* B_) {
  cplx* A = (cplx*)A_;
  cplx* B = (cplx*)B_;
  int64_t* piv = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!piv) return 1;
  for (int64_t c = 0; c < n; ++c) {
    int64_t p = c;
    double best = cabs(A[c * n + c]);
    for (int64_t r = c + 1; r < n; ++r) {
      double v = cabs(A[r * n + c]);
      if (v > best) {
        best = v;
        p = r;
      }
    }
    piv[c] = p;
    if (best == 0.0) {
      free(piv);
      return 2;
    }
    if (p != c) {
      for (int64_t j = 0; j < n; ++j) {
        cplx t = A[c * n + j];
        A[c * n + j] = A[p * n + j];
        A[p * n + j] = t;
      }
    }
    cplx inv = 1.0 / A[c * n + c];
#pragma omp parallel for schedule(static)
    for (int64_t r = c + 1; r < n; ++r) {
      cplx l = A[r * n + c] * inv;
      A[r * n + c] = l;
      for (int64_t j = c + 1; j < n; ++j) A[r * n + j] -= l * A[c * n + j];
    }
  }
  for (int q = 0; q < nrhs; ++q) {
    cplx* b = B + (int64_t)q * n;
    for (int64_t c = 0; c < n; ++c) {
      if (piv[c] != c) {
        cplx t = b[c];
        b[c] = b[piv[c]];
        b[piv[c]] = t;
      }
    }
    for (int64_t r = 0; r < n; ++r) {
      cplx s = b[r];
      for (int64_t j = 0; j < r; ++j) s -= A[r * n + j] * b[j];
      b[r] = s;
    }
    for (int64_t r = n - 1; r >= 0; --r) {
      cplx s = b[r];
      for (int64_t j = r + 1; j < n; ++j) s -= A[r * n + j] * b[j];
      b[r] = s / A[r * n + r];
    }
  }
  free(piv);
  return 0;
}
