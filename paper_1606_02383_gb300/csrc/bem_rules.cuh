// bem_rules.cuh -- the quadrature rules of the rule-defined collocation
// entries (Section 2.3): the 3-point rule R_0 on a flat triangle and its
// uniform refinement R_L (4^L pieces), in FP64 and in FP32 relative to the
// target, and the triangle loader from the stored FP64 geometry.  Shared by
// the correction build and the off-surface evaluation.
#pragma once
#include "bem_common.cuh"

// ------------------------------------------------------- FP64 quadrature --
struct Tri64 {
  double v[3][3];
  double n[3];
  double c[3];
  double area, h;
};

static __device__ __forceinline__ void kern64(const double* x, const double* y, const double* n, double w, double k,
                                       zd& s, zd& d) {
  double r3[3] = {y[0] - x[0], y[1] - x[1], y[2] - x[2]};
  double r = sqrt(r3[0] * r3[0] + r3[1] * r3[1] + r3[2] * r3[2]);
  double sn, cs;
  sincos(k * r, &sn, &cs);
  double g = w / (4.0 * BEM_PI * r);
  s.re += g * cs;
  s.im += g * sn;
  double rn = r3[0] * n[0] + r3[1] * n[1] + r3[2] * n[2];
  double f = w * rn / (4.0 * BEM_PI * r * r * r);
  // exp(ikr)(ikr - 1) = (-cs - kr sn) + i (kr cs - sn)
  d.re += f * (-cs - k * r * sn);
  d.im += f * (k * r * cs - sn);
}

// R_L: uniform subdivision L times, 3-point rule on each piece (iterative over 4^L pieces)
static __device__ void rule_refined(const double* x, const Tri64& t, int L, double k, zd& s, zd& d) {
  int npieces = 1 << (2 * L);
  double w = t.area / (3.0 * npieces);
  for (int piece = 0; piece < npieces; ++piece) {
    double a[3], b[3], c[3];
    for (int dd = 0; dd < 3; ++dd) {
      a[dd] = t.v[0][dd];
      b[dd] = t.v[1][dd];
      c[dd] = t.v[2][dd];
    }
    int code = piece;
    for (int lvl = 0; lvl < L; ++lvl) {
      int child = code & 3;
      code >>= 2;
      double ab[3], bc[3], ca[3];
      for (int dd = 0; dd < 3; ++dd) {
        ab[dd] = 0.5 * (a[dd] + b[dd]);
        bc[dd] = 0.5 * (b[dd] + c[dd]);
        ca[dd] = 0.5 * (c[dd] + a[dd]);
      }
      for (int dd = 0; dd < 3; ++dd) {
        if (child == 0) {
          b[dd] = ab[dd];
          c[dd] = ca[dd];
        } else if (child == 1) {
          a[dd] = ab[dd];
          c[dd] = bc[dd];
        } else if (child == 2) {
          a[dd] = ca[dd];
          b[dd] = bc[dd];
        } else {
          a[dd] = ab[dd];
          b[dd] = bc[dd];
          c[dd] = ca[dd];
        }
      }
    }
    const double b0 = 2.0 / 3.0, b1 = 1.0 / 6.0;
    for (int q = 0; q < 3; ++q) {
      double y[3];
      for (int dd = 0; dd < 3; ++dd)
        y[dd] = (q == 0 ? b0 : b1) * a[dd] + (q == 1 ? b0 : b1) * b[dd] + (q == 2 ? b0 : b1) * c[dd];
      kern64(x, y, t.n, w, k, s, d);
    }
  }
}

// FP32 versions for the mixed modes, with the triangle in coordinates
// relative to the target (so the point differences stay accurate in FP32)
struct Tri32 {
  float v[3][3];
  float n[3];
  float area;
};

static __device__ __forceinline__ void kern32(const float* y, const float* n, float w, float k, zf& s, zf& d) {
  const float r = sqrtf(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
  float sn, cs;
  sincosf(k * r, &sn, &cs);
  const float g = w / (4.0f * (float)BEM_PI * r);
  s.re += g * cs;
  s.im += g * sn;
  const float rn = y[0] * n[0] + y[1] * n[1] + y[2] * n[2];
  const float f = w * rn / (4.0f * (float)BEM_PI * r * r * r);
  d.re += f * (-cs - k * r * sn);
  d.im += f * (k * r * cs - sn);
}

// R_L on a target-relative triangle (same pieces and points as rule_refined)
static __device__ void rule_refined32(const Tri32& t, int L, float k, zf& s, zf& d) {
  const int npieces = 1 << (2 * L);
  const float w = t.area / (3.0f * npieces);
  for (int piece = 0; piece < npieces; ++piece) {
    float a[3], b[3], c[3];
    for (int dd = 0; dd < 3; ++dd) {
      a[dd] = t.v[0][dd];
      b[dd] = t.v[1][dd];
      c[dd] = t.v[2][dd];
    }
    int code = piece;
    for (int lvl = 0; lvl < L; ++lvl) {
      const int child = code & 3;
      code >>= 2;
      float ab[3], bc[3], ca[3];
      for (int dd = 0; dd < 3; ++dd) {
        ab[dd] = 0.5f * (a[dd] + b[dd]);
        bc[dd] = 0.5f * (b[dd] + c[dd]);
        ca[dd] = 0.5f * (c[dd] + a[dd]);
      }
      for (int dd = 0; dd < 3; ++dd) {
        if (child == 0) {
          b[dd] = ab[dd];
          c[dd] = ca[dd];
        } else if (child == 1) {
          a[dd] = ab[dd];
          c[dd] = bc[dd];
        } else if (child == 2) {
          a[dd] = ca[dd];
          b[dd] = bc[dd];
        } else {
          a[dd] = ab[dd];
          b[dd] = bc[dd];
          c[dd] = ca[dd];
        }
      }
    }
    const float b0 = 2.0f / 3.0f, b1 = 1.0f / 6.0f;
    for (int q = 0; q < 3; ++q) {
      float y[3];
      for (int dd = 0; dd < 3; ++dd)
        y[dd] = (q == 0 ? b0 : b1) * a[dd] + (q == 1 ? b0 : b1) * b[dd] + (q == 2 ? b0 : b1) * c[dd];
      kern32(y, t.n, w, k, s, d);
    }
  }
}

static __device__ void load_tri64(const double* __restrict__ qpt, const double* __restrict__ nrm,
                           const double* __restrict__ cent, const double* __restrict__ area,
                           const double* __restrict__ hmax, int j, Tri64& t) {
  // vertices from the quadrature points: q_a = c + (v_a - c)/2  =>  v_a = 2 q_a - c
  for (int d = 0; d < 3; ++d) {
    t.c[d] = cent[3 * j + d];
    t.n[d] = nrm[3 * j + d];
    for (int a = 0; a < 3; ++a) t.v[a][d] = 2.0 * qpt[9 * j + 3 * a + d] - t.c[d];
  }
  t.area = area[j];
  t.h = hmax[j];
}
