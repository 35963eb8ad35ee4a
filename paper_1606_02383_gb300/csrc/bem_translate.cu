// bem_translate.cu -- far-field operators of the fast multipole method, built in
// FP64 on the device at setup.
//
// Expansions (Section 2.3: "a low-frequency FMM is employed"; the paper gives
// no formulas, this is the standard Gegenbauer form).  With orthonormal
// spherical harmonics Y_nm = Pbar_n^|m|(cos theta) e^{i m phi} (associated
// Legendre functions without the Condon-Shortley phase, as in Section 2.2),
// regular and outgoing wave functions R_nm(v) = j_n(k|v|) Y_nm(v^),
// S_nm(v) = h_n(k|v|) Y_nm(v^), and for |y - c| < |x - c|
//     G(x - y) = i k sum_nm S_nm(x - c) conj(R_nm(y - c)).
// A multipole expansion about c is u(x) = sum M_nm S_nm(x - c) with
// M_nm = i k sum_j q_j conj(R_nm(y_j - c)); a local expansion about c' is
// u(x) = sum L_nm R_nm(x - c').
//
// Translations are written through Gaunt coefficients
//     Gaunt(n',m',n,m,l) = int conj(Y_n'm') Y_nm Y_l,m'-m dOmega
// (a 1-D Gauss-Legendre integral of three Pbar's, exact for these degrees):
//   M2L (c_s -> c_t, X = c_t - c_s):
//     T_{n'm',nm} = 4 pi i^{n'-n} sum_l i^l h_l(k|X|) conj(Y_l,m'-m(X^)) Gaunt
//   M2M (child c_c -> parent c_p, d = c_c - c_p):
//     T_{n'm',nm} = 4 pi i^{n'-n} sum_l (-i)^l j_l(k|d|) conj(Y_l,m'-m(d^)) Gaunt
//   L2L (parent c_p -> child c_c, e = c_c - c_p):
//     T_{n'm',nm} = 4 pi i^{n'-n} sum_l i^l j_l(k|e|) conj(Y_l,m'-m(e^)) Gaunt
// (from the plane-wave expansion exp(i k s.r) = 4 pi sum i^n j_n Y_nm(r^) conj(Y_nm(s))
// and Gegenbauer's addition theorem; the sum over l runs over
// |n-n'| <= l <= n+n', n+n'+l even, so each entry is a short sum of terms of
// one sign pattern and no cancellation between large terms occurs).
//
// Scaling: with s_n(l) = (k w_l)^n / (2n+1)!! (w_l the box width) the device
// stores M~ = M / s and L~ = L s, so every stored quantity is O(1) in FP32 at
// any frequency and box size; the scales are folded into the matrices and the
// P2M / L2P rows.
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>

#include "bem_common.cuh"

#define IDX(n, m) ((n) * (n) + (n) + (m))

// ------------------------------------------------------- special functions --
// Scaled spherical Bessel functions Jhat_n(x) = j_n(x) (2n+1)!! / x^n, n = 0..N.
// x < 1: power series in x^2; otherwise Miller's downward recurrence normalised
// by j_0 = sin x / x or j_1 = sin x/x^2 - cos x/x (whichever is larger).
__device__ void sph_jhat(double x, int N, double* out) {
  if (x < 1.0) {
    double x2h = -0.5 * x * x;
    for (int n = 0; n <= N; ++n) {
      double term = 1.0, sum = 1.0;
      for (int s = 1; s < 40; ++s) {
        term *= x2h / (s * (2.0 * n + 2.0 * s + 1.0));
        sum += term;
        if (fabs(term) < 1e-18 * fabs(sum)) break;
      }
      out[n] = sum;
    }
    return;
  }
  int M = max(N, (int)ceil(x)) + 60;
  double jp1 = 0.0, j = 1e-200;
  // out[] temporarily holds unnormalised j_n
  for (int n = M; n >= 1; --n) {
    double jm1 = (2.0 * n + 1.0) / x * j - jp1;
    jp1 = j;
    j = jm1;
    if (n - 1 <= N) out[n - 1] = j;
    if (n <= N) out[n] = jp1;
    if (fabs(j) > 1e200) {  // rescale everything kept so far
      j *= 1e-200;
      jp1 *= 1e-200;
      for (int q = n - 1; q <= N; ++q)
        if (q >= 0) out[q] *= 1e-200;
    }
  }
  double sn, cs;
  sincos(x, &sn, &cs);
  double j0 = sn / x, j1 = sn / (x * x) - cs / x;
  double scale = (fabs(j0) >= fabs(j1) || N < 1) ? j0 / out[0] : j1 / out[1];
  double fac = 1.0;  // (2n+1)!! / x^n
  for (int n = 0; n <= N; ++n) {
    if (n > 0) fac *= (2.0 * n + 1.0) / x;
    out[n] = out[n] * scale * fac;
  }
}

// j_n(x) and y_n(x), n = 0..N (x > 0)
__device__ void sph_jy(double x, int N, double* jn, double* yn) {
  sph_jhat(x, N, jn);
  double fac = 1.0;
  for (int n = 0; n <= N; ++n) {
    if (n > 0) fac *= x / (2.0 * n + 1.0);
    jn[n] *= fac;
  }
  double sn, cs;
  sincos(x, &sn, &cs);
  yn[0] = -cs / x;
  if (N >= 1) yn[1] = -cs / (x * x) - sn / x;
  for (int n = 1; n < N; ++n) yn[n + 1] = (2.0 * n + 1.0) / x * yn[n] - yn[n - 1];
}

// normalised associated Legendre Pbar_n^m(t), 0 <= m <= n <= N, stored at IDXP(n,m)
#define IDXP(n, m) ((n) * ((n) + 1) / 2 + (m))
__host__ __device__ inline void legendre_bar(double t, int N, double* P) {
  double st = sqrt(fmax(0.0, 1.0 - t * t));
  P[0] = 0.28209479177387814347;  // 1/sqrt(4 pi)
  for (int m = 1; m <= N; ++m) P[IDXP(m, m)] = sqrt((2.0 * m + 1.0) / (2.0 * m)) * st * P[IDXP(m - 1, m - 1)];
  for (int m = 0; m < N; ++m) P[IDXP(m + 1, m)] = sqrt(2.0 * m + 3.0) * t * P[IDXP(m, m)];
  for (int m = 0; m <= N; ++m)
    for (int n = m + 2; n <= N; ++n) {
      double a = sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
      double b = sqrt((((double)(n - 1) * (n - 1)) - (double)m * m) / (4.0 * (n - 1) * (n - 1) - 1.0));
      P[IDXP(n, m)] = a * (t * P[IDXP(n - 1, m)] - b * P[IDXP(n - 2, m)]);
    }
}

// ----------------------------------------------------------- Gaunt table --
// values[off[row*Pmax+col] + i] for the i-th admissible l of entry (row=n'm', col=nm)
__global__ void k_legendre_table(int Q, int N, const double* __restrict__ tq, double* tab) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  legendre_bar(tq[q], N, tab + (int64_t)q * ((N + 1) * (N + 2) / 2));
}

__global__ void k_gaunt(int pmax, int Q, int N, const double* __restrict__ wq, const double* __restrict__ tab,
                        const int64_t* __restrict__ off, double* vals) {
  int Pm = (pmax + 1) * (pmax + 1);
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)Pm * Pm) return;
  int row = (int)(e / Pm), col = (int)(e % Pm);
  int n1 = (int)floor(sqrt((double)row)), m1 = row - n1 * n1 - n1;
  int n = (int)floor(sqrt((double)col)), m = col - n * n - n;
  int mu = m1 - m;
  int lmin = max(abs(n - n1), abs(mu));
  if ((lmin + n + n1) & 1) ++lmin;
  int64_t o = off[e];
  int stride = (N + 1) * (N + 2) / 2;
  int am1 = abs(m1), am = abs(m), amu = abs(mu);
  for (int l = lmin, i = 0; l <= n + n1; l += 2, ++i) {
    double s = 0.0;
    for (int q = 0; q < Q; ++q) {
      const double* P = tab + (int64_t)q * stride;
      s += wq[q] * P[IDXP(n1, am1)] * P[IDXP(n, am)] * P[IDXP(l, amu)];
    }
    vals[o + i] = 2.0 * BEM_PI * s;
  }
}

// -------------------------------------------------------- translation mats --
struct MatJob {
  double v[3];   // translation vector
  int kind;      // 0 = M2L (h_l, i^l), 1 = M2M (j_l, (-i)^l), 2 = L2L (j_l, i^l)
  int p_out, p_in;
  int lev_out, lev_in;
  int64_t mat_off;
};

// per job: radial functions f_l and conj(Y_lmu(v^)) for l <= p_out + p_in
__global__ void k_mat_prep(const MatJob* __restrict__ jobs, int njobs, double k, int Lmax, double* fl_re, double* fl_im,
                           double* ylm_re, double* ylm_im, double* scratch) {
  int jb = blockIdx.x * blockDim.x + threadIdx.x;
  if (jb >= njobs) return;
  MatJob J = jobs[jb];
  int N = J.p_out + J.p_in;
  double r = sqrt(J.v[0] * J.v[0] + J.v[1] * J.v[1] + J.v[2] * J.v[2]);
  double* jn = scratch + (int64_t)jb * (4 * (Lmax + 2) + (Lmax + 1) * (Lmax + 2) / 2);
  double* yn = jn + (Lmax + 2);
  double* P = yn + (Lmax + 2);
  sph_jy(k * r, N, jn, yn);
  int64_t fo = (int64_t)jb * (Lmax + 1);
  for (int l = 0; l <= N; ++l) {
    fl_re[fo + l] = jn[l];
    fl_im[fo + l] = (J.kind == 0) ? yn[l] : 0.0;
  }
  double t = J.v[2] / r;
  double phi = atan2(J.v[1], J.v[0]);
  legendre_bar(t, N, P);
  int64_t yo = (int64_t)jb * (Lmax + 1) * (Lmax + 1);
  for (int l = 0; l <= N; ++l)
    for (int mu = -l; mu <= l; ++mu) {
      double pb = P[IDXP(l, abs(mu))];
      double s, c;
      sincos(mu * phi, &s, &c);
      ylm_re[yo + IDX(l, mu)] = pb * c;   // conj(Y_l,mu) = pb e^{-i mu phi}
      ylm_im[yo + IDX(l, mu)] = -pb * s;
    }
}

__device__ __forceinline__ double scale_n(double kw, int n) {  // (k w)^n / (2n+1)!!
  double s = 1.0;
  for (int q = 1; q <= n; ++q) s *= kw / (2.0 * q + 1.0);
  return s;
}

template <typename R>
__global__ void k_mat_fill(const MatJob* __restrict__ jobs, int job0, int pmax, double k, int Lmax,
                           const double* __restrict__ lev_w, const double* __restrict__ fl_re,
                           const double* __restrict__ fl_im, const double* __restrict__ ylm_re,
                           const double* __restrict__ ylm_im, const int64_t* __restrict__ goff,
                           const double* __restrict__ gval, R* mats, int* err) {
  int jb = job0 + blockIdx.y;
  MatJob J = jobs[jb];
  int Po = (J.p_out + 1) * (J.p_out + 1), Pi = (J.p_in + 1) * (J.p_in + 1);
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Po * Pi) return;
  int row = e / Pi, col = e % Pi;
  int n1 = (int)floor(sqrt((double)row)), m1 = row - n1 * n1 - n1;
  int n = (int)floor(sqrt((double)col)), m = col - n * n - n;
  int mu = m1 - m;
  int lmin = max(abs(n - n1), abs(mu));
  if ((lmin + n + n1) & 1) ++lmin;
  int Pm = (pmax + 1) * (pmax + 1);
  int64_t go = goff[(int64_t)row * Pm + col];
  int64_t fo = (int64_t)jb * (Lmax + 1);
  int64_t yo = (int64_t)jb * (Lmax + 1) * (Lmax + 1);
  zd acc = cmk(0.0, 0.0);
  for (int l = lmin, i = 0; l <= n + n1; l += 2, ++i) {
    zd c = (J.kind == 1) ? ipow(-l) : ipow(l);
    zd f = cmk(fl_re[fo + l], fl_im[fo + l]);
    zd y = cmk(ylm_re[yo + IDX(l, mu)], ylm_im[yo + IDX(l, mu)]);
    acc = acc + gval[go + i] * (c * f * y);
  }
  acc = (4.0 * BEM_PI) * (ipow(n1 - n) * acc);
  // scaled operator
  double kwo = k * lev_w[J.lev_out], kwi = k * lev_w[J.lev_in];
  double so = scale_n(kwo, n1), si = scale_n(kwi, n);
  double fac;
  if (J.kind == 0) fac = so * si;        // L~ = s L, M~ = M / s
  else if (J.kind == 1) fac = si / so;   // M~_p = (1/s_p) T s_c M~_c
  else fac = so / si;                    // L~_c = s_c T (1/s_p) L~_p
  acc = fac * acc;
  if (!isfinite(acc.re) || !isfinite(acc.im)) {
    atomicOr(err, BEM_DEVERR_OVERFLOW);
    acc = cmk(0.0, 0.0);
  }
  R* out = mats + 2 * (J.mat_off + (int64_t)row * Pi + col);
  out[0] = (R)acc.re;
  out[1] = (R)acc.im;
}

// ------------------------------------------------------- P2M / L2P rows --
// Solid harmonic S_nm(u) = |u|^n Y_nm(u^) and its derivative along dir, m >= 0
// via W_n^m = |u|^{n-m} Qbar_n^m(u_z/|u|) (a polynomial) times (u_x + i u_y)^m.
struct dual {
  double v, d;
};
__device__ __forceinline__ dual dmul(dual a, dual b) { return {a.v * b.v, a.v * b.d + a.d * b.v}; }

template <int PM>
__device__ void solid_harmonics(const double* u, const double* dir, int p, zd* S, zd* dS) {
  // W recurrences (duals), per m
  dual uz = {u[2], dir[2]};
  dual r2 = {u[0] * u[0] + u[1] * u[1] + u[2] * u[2], 2.0 * (u[0] * dir[0] + u[1] * dir[1] + u[2] * dir[2])};
  // xi^m (complex duals)
  zd xi = cmk(u[0], u[1]), dxi = cmk(dir[0], dir[1]);
  zd pw = cmk(1.0, 0.0), dpw = cmk(0.0, 0.0);
  double qmm = 0.28209479177387814347;  // Qbar_0^0
  for (int m = 0; m <= p; ++m) {
    if (m > 0) {
      qmm *= sqrt((2.0 * m + 1.0) / (2.0 * m));
      zd npw = pw * xi;
      zd ndpw = dpw * xi + pw * dxi;
      pw = npw;
      dpw = ndpw;
    }
    dual wm2 = {0.0, 0.0}, wm1 = {qmm, 0.0};
    for (int n = m; n <= p; ++n) {
      dual w;
      if (n == m) {
        w = wm1;
      } else if (n == m + 1) {
        double c = sqrt(2.0 * m + 3.0);
        w = {c * uz.v * wm1.v, c * (uz.d * wm1.v + uz.v * wm1.d)};
      } else {
        double a = sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
        double b = sqrt((((double)(n - 1) * (n - 1)) - (double)m * m) / (4.0 * (n - 1) * (n - 1) - 1.0));
        dual t1 = dmul(uz, wm1), t2 = dmul(r2, wm2);
        w = {a * (t1.v - b * t2.v), a * (t1.d - b * t2.d)};
      }
      if (n > m) {
        wm2 = wm1;
        wm1 = w;
      }
      zd val = w.v * pw;
      zd dval = w.d * pw + w.v * dpw;
      S[IDX(n, m)] = val;
      dS[IDX(n, m)] = dval;
      if (m > 0) {
        S[IDX(n, -m)] = conjc(val);
        dS[IDX(n, -m)] = conjc(dval);
      }
    }
  }
}

// order, box width and box centres of every leaf level, for the row builder
struct LevRows {
  int p[BEM_MAXLEV + 1];
  double w[BEM_MAXLEV + 1];
  const double* centre[BEM_MAXLEV + 1];
};

// one thread per (sorted) element, about the centre of the element's leaf
// with that leaf level's order; the rows start at complex offsets
// 2 row_off[j] (a: conj rows for S, then b: normal-derivative rows, P each)
// and row_off[j] (r: L2P rows).  Elements of leaves above level 2 have none.
template <typename R, int PM>
__global__ void k_p2m_l2p_rows(int64_t nt, LevRows lr, double k, const double* __restrict__ cent,
                               const double* __restrict__ qpt, const double* __restrict__ nrm,
                               const int* __restrict__ leaf_of, const unsigned char* __restrict__ leaf_lev,
                               const int64_t* __restrict__ row_off, int Pscr, R* rows_ab_base, R* rows_r_base,
                               double* scratch, int* err) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= nt) return;
  const int lvl = leaf_lev[j];
  if (lvl < 2) return;
  const int p = lr.p[lvl];
  const double w = lr.w[lvl];
  const int P = (p + 1) * (p + 1);
  zd* S = (zd*)(scratch + (int64_t)j * 4 * Pscr * 2 + 0);
  zd* dS = S + P;
  zd* A = dS + P;
  zd* B = A + P;
  double jh[PM + 3];
  int b = leaf_of[j];
  const double* bcentre = lr.centre[lvl];
  double c[3] = {bcentre[3 * b], bcentre[3 * b + 1], bcentre[3 * b + 2]};
  double nn[3] = {nrm[3 * j], nrm[3 * j + 1], nrm[3 * j + 2]};
  for (int e = 0; e < P; ++e) A[e] = B[e] = cmk(0.0, 0.0);
  // P2M rows: 4 pi i k sum_q conj(R~(y_q - c)) and its normal derivative
  for (int q = 0; q < 3; ++q) {
    double v[3], u[3];
    for (int d = 0; d < 3; ++d) {
      v[d] = qpt[9 * j + 3 * q + d] - c[d];
      u[d] = v[d] / w;
    }
    double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    sph_jhat(k * r, p + 1, jh);
    solid_harmonics<PM>(u, nn, p, S, dS);
    double vn = v[0] * nn[0] + v[1] * nn[1] + v[2] * nn[2];
    for (int n = 0; n <= p; ++n) {
      double dj = -jh[n + 1] * k * k * vn / (2.0 * n + 3.0);
      for (int m = -n; m <= n; ++m) {
        int e = IDX(n, m);
        zd Rt = jh[n] * S[e];
        zd dRt = dj * S[e] + (jh[n] / w) * dS[e];
        A[e] = A[e] + conjc(Rt);
        B[e] = B[e] + conjc(dRt);
      }
    }
  }
  zd fac = cmk(0.0, 4.0 * BEM_PI * k);
  R* ab = rows_ab_base + 4 * row_off[j];
  for (int e = 0; e < P; ++e) {
    zd a = fac * A[e], bb = fac * B[e];
    ab[2 * e] = (R)a.re;
    ab[2 * e + 1] = (R)a.im;
    ab[2 * (P + e)] = (R)bb.re;
    ab[2 * (P + e) + 1] = (R)bb.im;
    if (!isfinite(a.re + a.im + bb.re + bb.im)) atomicOr(err, BEM_DEVERR_OVERFLOW);
  }
  // L2P row: R~(x_i - c)
  {
    double v[3], u[3];
    for (int d = 0; d < 3; ++d) {
      v[d] = cent[3 * j + d] - c[d];
      u[d] = v[d] / w;
    }
    double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    sph_jhat(k * r, p, jh);
    solid_harmonics<PM>(u, nn, p, S, dS);
    R* rr = rows_r_base + 2 * row_off[j];
    for (int n = 0; n <= p; ++n)
      for (int m = -n; m <= n; ++m) {
        int e = IDX(n, m);
        zd Rt = jh[n] * S[e];
        rr[2 * e] = (R)Rt.re;
        rr[2 * e + 1] = (R)Rt.im;
      }
  }
}

// row length of every element: P of its leaf level rounded up to even (0 above level 2)
__global__ void k_row_len(int64_t nt, const unsigned char* __restrict__ leaf_lev, LevTab lt, int64_t* len) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= nt) return;
  const int P = lt.P[leaf_lev[j]];
  len[j] = (P + 1) & ~1;
}

__global__ void k_pairs_to_offsets(int np, const int* __restrict__ src_box, const int* __restrict__ dst_box,
                                   int64_t src_base, int Psrc, int64_t dst_base, int Pdst, int* src_off, int* dst_off) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  src_off[i] = (int)(src_base + (int64_t)src_box[i] * Psrc);
  dst_off[i] = (int)(dst_base + (int64_t)dst_box[i] * Pdst);
}

// all children of one level as (child, parent, reflection flags) pairs: the
// canonical child offset is (+w/2, +w/2, +w/2); an axis whose octant bit is 0
// points the other way, so its flag bit is set
__global__ void k_octant_pairs(int nchild_boxes, const uint32_t* __restrict__ ckey, const int* __restrict__ cparent,
                               int* child_box, int* parent_box, unsigned char* flags) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nchild_boxes) return;
  child_box[c] = c;
  parent_box[c] = cparent[c];
  flags[c] = (unsigned char)((~ckey[c]) & 7u);
}

// move V-list pairs from per-offset blocks into per-canonical-offset blocks
// blk[i] = (old start, new start, count, flags)
__global__ void k_regroup(const int4* __restrict__ blk, const int* __restrict__ src_in, const int* __restrict__ dst_in,
                          int* src_out, int* dst_out, unsigned char* flags) {
  int4 B = blk[blockIdx.x];
  for (int i = threadIdx.x; i < B.z; i += blockDim.x) {
    src_out[B.y + i] = src_in[B.x + i];
    dst_out[B.y + i] = dst_in[B.x + i];
    flags[B.y + i] = (unsigned char)B.w;
  }
}

// ------------------------------------------------------------------ host --
static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Order of one level (Section 3: truncation "numerically determined" so the
// error stays below the tolerance).  Two terms: the high-frequency rule
// p = kd + c (d0)^(2/3) (kd)^(1/3) (d the box diameter, d0 = -log10 eps) and a
// low-frequency floor 1.6 d0 + 1.  The constants were calibrated on the
// 327,680-triangle sphere at ka = 20 and a 20,480-triangle sphere at ka = 5,
// against the FP64 oracle, for random densities and for smooth (plane-wave)
// single- and double-layer densities: the leaf order sets the error, the
// coarse-level orders mostly set the cost.
static int order_for_level(const bem_handle* h, int l, double w) {
  if (h->p_level[l] > 0) return h->p_level[l];
  if (h->fixed_p > 0) return h->fixed_p;
  double d0 = -std::log10(std::max(h->eps, 1e-15));
  double kd = h->k * std::sqrt(3.0) * w;
  double p_hf = kd + 1.0 * std::pow(d0, 2.0 / 3.0) * std::cbrt(std::max(kd, 1e-30));
  double p_lf = 1.6 * d0 + 1.0;
  int p = (int)std::ceil(std::max(p_hf, p_lf) - 1e-9);
  return std::min(std::max(p, h->p_min), h->p_max);
}

static void gl_nodes(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(BEM_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 200; ++it) {
      double p0 = 1.0, p1 = z;
      for (int m = 2; m <= n; ++m) {
        double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int m = 2; m <= n; ++m) {
      double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// tile jobs: groups with many pairs use 64 x 64 output tiles, small groups 128 x 16
static int make_jobs(bem_handle* h, GroupedOp& op, cudaStream_t s) {
  std::vector<int4> ja, jb;
  op.flops = 0;
  for (int g = 0; g < op.ngroups; ++g) {
    int np = op.pair_start[g + 1] - op.pair_start[g];
    op.flops += 8LL * op.rows[g] * op.cols[g] * np;
    bool wide = np >= 40;
    int TN = wide ? 64 : 16, TM = wide ? 64 : 128;
    const int KS = 128;  // K slice per job (matches the kernel)
    for (int p0 = 0; p0 < np; p0 += TN)
      for (int r0 = 0; r0 < op.rows[g]; r0 += TM)
        for (int kt = 0; kt * KS < op.cols[g]; ++kt)
          (wide ? ja : jb).push_back(make_int4(g, op.pair_start[g] + p0, std::min(TN, np - p0) | (kt << 8), r0));
  }
  op.njobsA = (int)ja.size();
  op.njobsB = (int)jb.size();
  BEM_TRY(bem_alloc(h, &op.d_jobsA, std::max<size_t>(ja.size(), 1)));
  BEM_TRY(bem_alloc(h, &op.d_jobsB, std::max<size_t>(jb.size(), 1)));
  BEM_TRY(bem_alloc(h, &op.d_group_rows, std::max(op.ngroups, 1)));
  BEM_TRY(bem_alloc(h, &op.d_group_cols, std::max(op.ngroups, 1)));
  BEM_TRY(bem_alloc(h, &op.d_group_mat, std::max(op.ngroups, 1)));
  if (!ja.empty()) BEM_CUDA(cudaMemcpyAsync(op.d_jobsA, ja.data(), ja.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
  if (!jb.empty()) BEM_CUDA(cudaMemcpyAsync(op.d_jobsB, jb.data(), jb.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
  if (op.ngroups) {
    BEM_CUDA(cudaMemcpyAsync(op.d_group_rows, op.rows.data(), op.ngroups * sizeof(int), cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyAsync(op.d_group_cols, op.cols.data(), op.ngroups * sizeof(int), cudaMemcpyHostToDevice, s));
    BEM_CUDA(
        cudaMemcpyAsync(op.d_group_mat, op.mat_off.data(), op.ngroups * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  }
  BEM_CUDA(cudaStreamSynchronize(s));  // host vectors are temporaries
  return BEM_OK;
}

int bem_build_far_field(bem_handle* h, cudaStream_t s) {
  int L = h->L;
  int64_t nt = h->nt;
  // orders and expansion layout
  int pmax = 0;
  h->exp_total = 0;
  for (int l = 2; l <= L; ++l) {
    LevelInfo& lv = h->lev[l];
    lv.p = order_for_level(h, l, lv.w);
    lv.P = (lv.p + 1) * (lv.p + 1);
    lv.exp_base = h->exp_total;
    h->exp_total += (int64_t)lv.nbox * lv.P;
    pmax = std::max(pmax, lv.p);
  }
  if (h->exp_total > 2000000000LL) return bem_fail(BEM_ERR_UNSUPPORTED, "expansion storage exceeds 32-bit offsets");
  BEM_TRY(bem_build_wx_tables(h, s));
  h->w_evals = h->x_evals = 0;
  for (int l = 2; l <= L; ++l) {
    h->w_evals += h->w_tp[l] * h->lev[l].P;
    h->x_evals += h->x_pts[l] * h->lev[l].P;
  }
  bool f64 = bem_is_fp64(h);
  size_t csz = f64 ? 2 * sizeof(double) : 2 * sizeof(float);
  int Pm = (pmax + 1) * (pmax + 1);

  int* leaf_of = h->leaf_of;  // leaf membership (built with the tree)

  // ---- groups: M2L (from the V-lists), M2M/L2L (octants) ----
  std::vector<MatJob> mj;
  int64_t mat_len = 0;
  auto add_mat = [&](int kind, const double* v, int p_out, int p_in, int lo, int li) {
    MatJob J;
    J.v[0] = v[0];
    J.v[1] = v[1];
    J.v[2] = v[2];
    J.kind = kind;
    J.p_out = p_out;
    J.p_in = p_in;
    J.lev_out = lo;
    J.lev_in = li;
    J.mat_off = mat_len;
    mat_len += (int64_t)(p_out + 1) * (p_out + 1) * (p_in + 1) * (p_in + 1);
    mj.push_back(J);
    return J.mat_off;
  };
  for (int l = 2; l <= L; ++l) {
    GroupedOp& op = h->m2l[l];
    LevelInfo& lv = h->lev[l];
    // canonical offset (|dx|, |dy|, |dz|) and reflection flags of every code group
    std::vector<int> canon_of(op.ngroups), flag_of(op.ngroups);
    std::vector<int> ccount(343, 0);
    for (int g = 0; g < op.ngroups; ++g) {
      int o = op.codes[g];
      int dx = o / 49 - 3, dy = (o / 7) % 7 - 3, dz = o % 7 - 3;
      canon_of[g] = (std::abs(dx) + 3) * 49 + (std::abs(dy) + 3) * 7 + (std::abs(dz) + 3);
      flag_of[g] = (dx < 0 ? 1 : 0) | (dy < 0 ? 2 : 0) | (dz < 0 ? 4 : 0);
      ccount[canon_of[g]] += op.pair_start[g + 1] - op.pair_start[g];
    }
    std::vector<int> cstart(344, 0);
    for (int c = 0; c < 343; ++c) cstart[c + 1] = cstart[c] + ccount[c];
    std::vector<int4> blk;
    std::vector<int> cur(cstart.begin(), cstart.end() - 1);
    for (int g = 0; g < op.ngroups; ++g) {
      int cnt = op.pair_start[g + 1] - op.pair_start[g];
      blk.push_back(make_int4(op.pair_start[g], cur[canon_of[g]], cnt, flag_of[g]));
      cur[canon_of[g]] += cnt;
    }
    int np = op.npairs;
    int *src2, *dst2;
    int4* dblk;
    BEM_TRY(bem_alloc(h, &src2, std::max(np, 1)));
    BEM_TRY(bem_alloc(h, &dst2, std::max(np, 1)));
    BEM_TRY(bem_alloc(h, &op.d_flags, std::max(np, 1)));
    if (!blk.empty()) {
      BEM_CUDA(cudaMallocAsync((void**)&dblk, blk.size() * sizeof(int4), s));
      BEM_CUDA(cudaMemcpyAsync(dblk, blk.data(), blk.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
      k_regroup<<<(unsigned)blk.size(), 128, 0, s>>>(dblk, op.d_src_off, op.d_dst_off, src2, dst2, op.d_flags);
      BEM_CUDA(cudaGetLastError());
      BEM_CUDA(cudaStreamSynchronize(s));
      BEM_CUDA(cudaFreeAsync(dblk, s));
    }
    op.d_src_off = src2;
    op.d_dst_off = dst2;
    op.ngroups = 0;
    op.pair_start.clear();
    op.rows.clear();
    op.cols.clear();
    op.mat_off.clear();
    for (int c = 0; c < 343; ++c) {
      if (ccount[c] == 0) continue;
      int dx = c / 49 - 3, dy = (c / 7) % 7 - 3, dz = c % 7 - 3;
      double v[3] = {dx * lv.w, dy * lv.w, dz * lv.w};  // X = c_t - c_s (canonical)
      op.pair_start.push_back(cstart[c]);
      op.rows.push_back(lv.P);
      op.cols.push_back(lv.P);
      op.mat_off.push_back(add_mat(0, v, lv.p, lv.p, l, l));
      ++op.ngroups;
    }
    op.pair_start.push_back(np);
    if (np > 0)
      k_pairs_to_offsets<<<nblk(np, 256), 256, 0, s>>>(np, op.d_src_off, op.d_dst_off, lv.exp_base, lv.P,
                                                       lv.exp_base, lv.P, op.d_src_off, op.d_dst_off);
    BEM_CUDA(cudaGetLastError());
    BEM_TRY(make_jobs(h, op, s));
  }
  for (int l = 2; l < L; ++l) {
    // children at level l+1, parents at level l; one canonical matrix each way
    LevelInfo& pv = h->lev[l];
    LevelInfo& cv = h->lev[l + 1];
    int *cb, *pb;
    unsigned char* fl;
    BEM_CUDA(cudaMallocAsync((void**)&cb, std::max(cv.nbox, 1) * sizeof(int), s));
    BEM_CUDA(cudaMallocAsync((void**)&pb, std::max(cv.nbox, 1) * sizeof(int), s));
    BEM_CUDA(cudaMallocAsync((void**)&fl, std::max(cv.nbox, 1), s));
    k_octant_pairs<<<nblk(cv.nbox, 256), 256, 0, s>>>(cv.nbox, cv.key, cv.parent, cb, pb, fl);
    BEM_CUDA(cudaGetLastError());
    // only tree boxes take part (children of internal boxes): compact the pairs
    int ncp = cv.nbox;
    {
      std::vector<int> hcb(cv.nbox), hpb(cv.nbox);
      std::vector<unsigned char> hfl(cv.nbox), hin(cv.nbox);
      BEM_CUDA(cudaMemcpyAsync(hcb.data(), cb, cv.nbox * sizeof(int), cudaMemcpyDeviceToHost, s));
      BEM_CUDA(cudaMemcpyAsync(hpb.data(), pb, cv.nbox * sizeof(int), cudaMemcpyDeviceToHost, s));
      BEM_CUDA(cudaMemcpyAsync(hfl.data(), fl, cv.nbox, cudaMemcpyDeviceToHost, s));
      BEM_CUDA(cudaMemcpyAsync(hin.data(), cv.intree, cv.nbox, cudaMemcpyDeviceToHost, s));
      BEM_CUDA(cudaStreamSynchronize(s));
      ncp = 0;
      for (int c = 0; c < cv.nbox; ++c)
        if (hin[c]) {
          hcb[ncp] = hcb[c];
          hpb[ncp] = hpb[c];
          hfl[ncp] = hfl[c];
          ++ncp;
        }
      if (ncp > 0) {
        BEM_CUDA(cudaMemcpyAsync(cb, hcb.data(), ncp * sizeof(int), cudaMemcpyHostToDevice, s));
        BEM_CUDA(cudaMemcpyAsync(pb, hpb.data(), ncp * sizeof(int), cudaMemcpyHostToDevice, s));
        BEM_CUDA(cudaMemcpyAsync(fl, hfl.data(), ncp, cudaMemcpyHostToDevice, s));
      }
      BEM_CUDA(cudaStreamSynchronize(s));
    }
    double hw = 0.5 * cv.w;
    double v[3] = {hw, hw, hw};  // canonical c_child - c_parent
    GroupedOp* ops[2] = {&h->m2m[l], &h->l2l[l]};
    for (int which = 0; which < 2; ++which) {
      GroupedOp& op = *ops[which];
      op.npairs = ncp;
      op.ngroups = ncp > 0 ? 1 : 0;
      op.pair_start = ncp > 0 ? std::vector<int>{0, ncp} : std::vector<int>{0};
      if (which == 0) {
        op.rows = {pv.P};
        op.cols = {cv.P};
        op.mat_off = {add_mat(1, v, pv.p, cv.p, l, l + 1)};
      } else {
        op.rows = {cv.P};
        op.cols = {pv.P};
        op.mat_off = {add_mat(2, v, cv.p, pv.p, l + 1, l)};
      }
      BEM_TRY(bem_alloc(h, &op.d_src_off, std::max(ncp, 1)));
      BEM_TRY(bem_alloc(h, &op.d_dst_off, std::max(ncp, 1)));
      BEM_TRY(bem_alloc(h, &op.d_flags, std::max(ncp, 1)));
      if (ncp > 0) {
        BEM_CUDA(cudaMemcpyAsync(op.d_flags, fl, ncp, cudaMemcpyDeviceToDevice, s));
        if (which == 0)
          k_pairs_to_offsets<<<nblk(ncp, 256), 256, 0, s>>>(ncp, cb, pb, cv.exp_base, cv.P, pv.exp_base, pv.P,
                                                            op.d_src_off, op.d_dst_off);
        else
          k_pairs_to_offsets<<<nblk(ncp, 256), 256, 0, s>>>(ncp, pb, cb, pv.exp_base, pv.P, cv.exp_base, cv.P,
                                                            op.d_src_off, op.d_dst_off);
        BEM_CUDA(cudaGetLastError());
      }
      BEM_TRY(make_jobs(h, op, s));
    }
    BEM_CUDA(cudaStreamSynchronize(s));
    BEM_CUDA(cudaFreeAsync(cb, s));
    BEM_CUDA(cudaFreeAsync(pb, s));
    BEM_CUDA(cudaFreeAsync(fl, s));
  }

  // ---- Gaunt table for n, n' <= pmax ----
  int Lmax = 2 * pmax;
  std::vector<int64_t> goff((size_t)Pm * Pm);
  int64_t gtot = 0;
  for (int row = 0; row < Pm; ++row) {
    int n1 = (int)std::floor(std::sqrt((double)row)), m1 = row - n1 * n1 - n1;
    for (int col = 0; col < Pm; ++col) {
      int n = (int)std::floor(std::sqrt((double)col)), m = col - n * n - n;
      int lmin = std::max(std::abs(n - n1), std::abs(m1 - m));
      if ((lmin + n + n1) & 1) ++lmin;
      goff[(size_t)row * Pm + col] = gtot;
      if (lmin <= n + n1) gtot += (n + n1 - lmin) / 2 + 1;
    }
  }
  int Q = 2 * pmax + 2;
  std::vector<double> tq, wq;
  gl_nodes(Q, tq, wq);
  double *d_tq, *d_wq, *d_tab, *d_gval;
  int64_t* d_goff;
  int tabstride = (Lmax + 1) * (Lmax + 2) / 2;
  BEM_CUDA(cudaMallocAsync((void**)&d_tq, Q * sizeof(double), s));
  BEM_CUDA(cudaMallocAsync((void**)&d_wq, Q * sizeof(double), s));
  BEM_CUDA(cudaMallocAsync((void**)&d_tab, (size_t)Q * tabstride * sizeof(double), s));
  BEM_CUDA(cudaMallocAsync((void**)&d_gval, std::max<int64_t>(gtot, 1) * sizeof(double), s));
  BEM_CUDA(cudaMallocAsync((void**)&d_goff, goff.size() * sizeof(int64_t), s));
  BEM_CUDA(cudaMemcpyAsync(d_tq, tq.data(), Q * sizeof(double), cudaMemcpyHostToDevice, s));
  BEM_CUDA(cudaMemcpyAsync(d_wq, wq.data(), Q * sizeof(double), cudaMemcpyHostToDevice, s));
  BEM_CUDA(cudaMemcpyAsync(d_goff, goff.data(), goff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  k_legendre_table<<<nblk(Q, 64), 64, 0, s>>>(Q, Lmax, d_tq, d_tab);
  k_gaunt<<<nblk((int64_t)Pm * Pm, 128), 128, 0, s>>>(pmax, Q, Lmax, d_wq, d_tab, d_goff, d_gval);
  BEM_CUDA(cudaGetLastError());

  // ---- translation matrices ----
  h->mats_len = mat_len;
  if (f64) {
    double* m;
    BEM_TRY(bem_alloc(h, &m, 2 * std::max<int64_t>(mat_len, 1)));
    h->mats = m;
  } else {
    float* m;
    BEM_TRY(bem_alloc(h, &m, 2 * std::max<int64_t>(mat_len, 1)));
    h->mats = m;
  }
  int nj = (int)mj.size();
  if (nj > 0) {
    MatJob* d_jobs;
    double *fl_re, *fl_im, *y_re, *y_im, *scr, *d_levw;
    BEM_CUDA(cudaMallocAsync((void**)&d_jobs, nj * sizeof(MatJob), s));
    BEM_CUDA(cudaMallocAsync((void**)&fl_re, (size_t)nj * (Lmax + 1) * sizeof(double), s));
    BEM_CUDA(cudaMallocAsync((void**)&fl_im, (size_t)nj * (Lmax + 1) * sizeof(double), s));
    BEM_CUDA(cudaMallocAsync((void**)&y_re, (size_t)nj * (Lmax + 1) * (Lmax + 1) * sizeof(double), s));
    BEM_CUDA(cudaMallocAsync((void**)&y_im, (size_t)nj * (Lmax + 1) * (Lmax + 1) * sizeof(double), s));
    BEM_CUDA(cudaMallocAsync((void**)&scr, (size_t)nj * (4 * (Lmax + 2) + tabstride) * sizeof(double), s));
    BEM_CUDA(cudaMallocAsync((void**)&d_levw, (BEM_MAXLEV + 1) * sizeof(double), s));
    double levw[BEM_MAXLEV + 1];
    for (int l = 0; l <= BEM_MAXLEV; ++l) levw[l] = h->root_w / (1 << l);
    BEM_CUDA(cudaMemcpyAsync(d_levw, levw, sizeof(levw), cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyAsync(d_jobs, mj.data(), nj * sizeof(MatJob), cudaMemcpyHostToDevice, s));
    k_mat_prep<<<nblk(nj, 64), 64, 0, s>>>(d_jobs, nj, h->k, Lmax, fl_re, fl_im, y_re, y_im, scr);
    BEM_CUDA(cudaGetLastError());
    int maxPP = Pm * Pm;
    for (int j0 = 0; j0 < nj; j0 += 32768) {
      dim3 grid(nblk(maxPP, 128), std::min(32768, nj - j0));
      if (f64)
        k_mat_fill<double><<<grid, 128, 0, s>>>(d_jobs, j0, pmax, h->k, Lmax, d_levw, fl_re, fl_im, y_re, y_im, d_goff,
                                                d_gval, (double*)h->mats, h->d_err);
      else
        k_mat_fill<float><<<grid, 128, 0, s>>>(d_jobs, j0, pmax, h->k, Lmax, d_levw, fl_re, fl_im, y_re, y_im, d_goff,
                                               d_gval, (float*)h->mats, h->d_err);
      BEM_CUDA(cudaGetLastError());
    }
    BEM_CUDA(cudaStreamSynchronize(s));
    BEM_CUDA(cudaFreeAsync(d_jobs, s));
    BEM_CUDA(cudaFreeAsync(fl_re, s));
    BEM_CUDA(cudaFreeAsync(fl_im, s));
    BEM_CUDA(cudaFreeAsync(y_re, s));
    BEM_CUDA(cudaFreeAsync(y_im, s));
    BEM_CUDA(cudaFreeAsync(scr, s));
    BEM_CUDA(cudaFreeAsync(d_levw, s));
  }
  BEM_CUDA(cudaFreeAsync(d_tq, s));
  BEM_CUDA(cudaFreeAsync(d_wq, s));
  BEM_CUDA(cudaFreeAsync(d_tab, s));
  BEM_CUDA(cudaFreeAsync(d_gval, s));
  BEM_CUDA(cudaFreeAsync(d_goff, s));

  for (int l = 2; l <= L; ++l) h->m2l[l].mats_base = h->mats;
  for (int l = 2; l < L; ++l) {
    h->m2m[l].mats_base = h->mats;
    h->l2l[l].mats_base = h->mats;
  }
  // ---- tensor-core packing of every grouped operator (mixed mode) ----
  if (!f64) {
    for (int l = 2; l <= L; ++l) BEM_TRY(bem_build_tc(h, h->m2l[l], l, s));
    for (int l = 2; l < L; ++l) {
      h->m2m[l].upward = 1;
      BEM_TRY(bem_build_tc(h, h->m2m[l], l + 1, s));
      BEM_TRY(bem_build_tc(h, h->l2l[l], l, s));
    }
  }

  // ---- P2M / L2P rows of every element, about its leaf's centre ----
  // row offsets: P of the element's leaf level rounded up to even (16-byte
  // aligned rows), prefix-summed
  LevRows lr;
  int PLmax = 0;
  for (int l = 0; l <= BEM_MAXLEV; ++l) {
    const bool has = l >= 2 && l <= L;
    lr.p[l] = has ? h->lev[l].p : 0;
    lr.w[l] = has ? h->lev[l].w : 0.0;
    lr.centre[l] = has ? h->lev[l].centre : nullptr;
    if (has && h->lev[l].nleaf > 0) {
      if (h->lev[l].p > 60) return bem_fail(BEM_ERR_UNSUPPORTED, "leaf order above 60");
      PLmax = std::max(PLmax, h->lev[l].P);
    }
  }
  {
    LevTab lt = bem_levtab(h);
    int64_t* len;
    BEM_CUDA(cudaMallocAsync((void**)&len, nt * sizeof(int64_t), s));
    k_row_len<<<nblk(nt, 256), 256, 0, s>>>(nt, h->leaf_lev, lt, len);
    BEM_TRY(bem_alloc(h, &h->row_off, nt));
    size_t tbs = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, tbs, len, h->row_off, (int)nt, s);
    void* tsc;
    BEM_CUDA(cudaMallocAsync(&tsc, tbs, s));
    BEM_CUDA(cub::DeviceScan::ExclusiveSum(tsc, tbs, len, h->row_off, (int)nt, s));
    int64_t last[2] = {0, 0};
    BEM_CUDA(cudaMemcpyAsync(&last[0], h->row_off + nt - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaMemcpyAsync(&last[1], len + nt - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    h->row_total = last[0] + last[1];
    BEM_CUDA(cudaFreeAsync(tsc, s));
    BEM_CUDA(cudaFreeAsync(len, s));
  }
  const int64_t rt = std::max<int64_t>(h->row_total, 2);
  if (f64) {
    double *ab, *r;
    BEM_TRY(bem_alloc(h, &ab, (size_t)rt * 2 * 2));
    BEM_TRY(bem_alloc(h, &r, (size_t)rt * 2));
    h->p2m_rows = ab;
    h->l2p_rows = r;
  } else {
    float *ab, *r;
    BEM_TRY(bem_alloc(h, &ab, (size_t)rt * 2 * 2));
    BEM_TRY(bem_alloc(h, &r, (size_t)rt * 2));
    h->p2m_rows = ab;
    h->l2p_rows = r;
  }
  const int64_t chunk = 1 << 16;
  double* scr;
  BEM_CUDA(cudaMallocAsync((void**)&scr, (size_t)chunk * 4 * std::max(PLmax, 1) * 2 * sizeof(double), s));
  for (int64_t j0 = 0; j0 < nt && PLmax > 0; j0 += chunk) {
    int64_t cnt = std::min(chunk, nt - j0);
    // the kernel indexes scratch by its own element index, so offset pointers per chunk
    if (f64)
      k_p2m_l2p_rows<double, 64><<<nblk(cnt, 64), 64, 0, s>>>(
          cnt, lr, h->k, h->cent + 3 * j0, h->qpt + 9 * j0, h->nrm + 3 * j0, leaf_of + j0, h->leaf_lev + j0,
          h->row_off + j0, PLmax, (double*)h->p2m_rows, (double*)h->l2p_rows, scr, h->d_err);
    else
      k_p2m_l2p_rows<float, 64><<<nblk(cnt, 64), 64, 0, s>>>(
          cnt, lr, h->k, h->cent + 3 * j0, h->qpt + 9 * j0, h->nrm + 3 * j0, leaf_of + j0, h->leaf_lev + j0,
          h->row_off + j0, PLmax, (float*)h->p2m_rows, (float*)h->l2p_rows, scr, h->d_err);
    BEM_CUDA(cudaGetLastError());
  }
  BEM_CUDA(cudaStreamSynchronize(s));
  BEM_CUDA(cudaFreeAsync(scr, s));
  (void)csz;
  return bem_check_device_error(h, s);
}

// ------------------------------------------------------- adjoint operators --
// Plain transpose (no conjugation) of every group matrix: out[c][r] = in[r][c].
template <typename R>
__global__ void k_transpose_group(const R* __restrict__ in, R* __restrict__ out, int rows, int cols, int64_t off) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * cols) return;
  int r = (int)(e / cols), c = (int)(e % cols);
  out[2 * (off + (int64_t)c * rows + r)] = in[2 * (off + e)];
  out[2 * (off + (int64_t)c * rows + r) + 1] = in[2 * (off + e) + 1];
}

// The transpose of a grouped operator: same pairs with source and destination
// swapped, transposed matrices, same reflection flags ((Q T Q)^T = Q T^T Q).
static int make_transposed(bem_handle* h, const GroupedOp& op, GroupedOp& t, int src_level, cudaStream_t s) {
  t.ngroups = op.ngroups;
  t.rows = op.cols;
  t.cols = op.rows;
  t.mat_off = op.mat_off;
  t.pair_start = op.pair_start;
  t.npairs = op.npairs;
  t.d_src_off = op.d_dst_off;
  t.d_dst_off = op.d_src_off;
  t.d_flags = op.d_flags;
  t.mats_base = h->mats_T;
  bool f64 = bem_is_fp64(h);
  for (int g = 0; g < op.ngroups; ++g) {
    int64_t n = (int64_t)op.rows[g] * op.cols[g];
    if (f64)
      k_transpose_group<double><<<nblk(n, 256), 256, 0, s>>>((const double*)h->mats, (double*)h->mats_T, op.rows[g],
                                                             op.cols[g], op.mat_off[g]);
    else
      k_transpose_group<float><<<nblk(n, 256), 256, 0, s>>>((const float*)h->mats, (float*)h->mats_T, op.rows[g],
                                                            op.cols[g], op.mat_off[g]);
    BEM_CUDA(cudaGetLastError());
  }
  BEM_TRY(make_jobs(h, t, s));
  if (!f64) BEM_TRY(bem_build_tc(h, t, src_level, s));
  return BEM_OK;
}

int bem_build_adjoint(bem_handle* h, cudaStream_t s) {
  if (h->adj_ready) return BEM_OK;
  int64_t nt = h->nt;
  BEM_TRY(bem_alloc(h, &h->uv, (size_t)nt * h->nrhs_max));
  if (bem_is_fmm(h) && h->L >= 2) {
    if (bem_is_fp64(h)) {
      double* m;
      BEM_TRY(bem_alloc(h, &m, 2 * std::max<int64_t>(h->mats_len, 1)));
      h->mats_T = m;
    } else {
      float* m;
      BEM_TRY(bem_alloc(h, &m, 2 * std::max<int64_t>(h->mats_len, 1)));
      h->mats_T = m;
    }
    for (int l = 2; l <= h->L; ++l) BEM_TRY(make_transposed(h, h->m2l[l], h->m2l_T[l], l, s));
    for (int l = 2; l < h->L; ++l) {
      BEM_TRY(make_transposed(h, h->m2m[l], h->m2m_T[l], l, s));      // parent level -> children
      BEM_TRY(make_transposed(h, h->l2l[l], h->l2l_T[l], l + 1, s));  // children -> parent level
    }
  }
  BEM_TRY(bem_build_corr_transpose(h, s));
  BEM_CUDA(cudaStreamSynchronize(s));
  h->adj_ready = true;
  return BEM_OK;
}
