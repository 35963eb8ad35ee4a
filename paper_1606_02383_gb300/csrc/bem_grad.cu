// bem_grad.cu -- derivative of a real loss with respect to the wavenumber k.
//
// The operator A(k) = 1/2 I - D(k) on x plus S(k) on y depends on k only
// through the kernels (Section 2.3, G = exp(ikr)/(4 pi r)):
//   dG/dk            = i exp(ikr) / (4 pi)
//   d(dG/dn_y)/dk    = -k exp(ikr) (y - x).n / (4 pi r)
// both smooth, and through the exact self term,
//   dS_ii/dk = (1/4 pi) int_T i exp(ikr) dA.
// For an upstream gradient g (PyTorch convention for complex outputs) the loss
// derivative is dk = sum_rhs Re < g, (dA/dk) u >.  The regular rule R_0 over
// all pairs is summed by the target-major pass of the vertex gradient
// (bem_grad_vertices.cu: FP64 in the FP64 modes, FP32 with split coordinates
// otherwise); the near-singular / self corrections add d/dk of (rule R_L or
// exact) - R_0 for the pairs of the correction matrix: here when dL/dk alone
// is asked for, otherwise inside the vertex gradient's correction and self
// kernels on the same quadrature points.
#include "bem_common.cuh"

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// unweighted densities (y, x) and g in octree order, FP64
template <typename Rin>
__global__ void k_grad_prologue(int64_t nt, int nrhs, const int* __restrict__ perm, const Rin* __restrict__ g,
                                const Rin* __restrict__ x, const Rin* __restrict__ y, double4* yx, double2* gs) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nt) return;
  int64_t o = perm[s];
  for (int r = 0; r < nrhs; ++r) {
    int64_t io = 2 * ((int64_t)r * nt + o);
    yx[(int64_t)r * nt + s] = make_double4(y ? (double)y[io] : 0.0, y ? (double)y[io + 1] : 0.0,
                                           x ? (double)x[io] : 0.0, x ? (double)x[io + 1] : 0.0);
    gs[(int64_t)r * nt + s] = make_double2((double)g[io], (double)g[io + 1]);
  }
}

// sin/cos in the precision of the evaluation
__device__ __forceinline__ void gsc(float a, float* s, float* c) { sincosf(a, s, c); }
__device__ __forceinline__ void gsc(double a, double* s, double* c) { sincos(a, s, c); }

// d/dk of one point of weight wq: returns (dS, dD) contributions at target x
template <typename R>
__device__ __forceinline__ void dk_point(const R* x, const R* y, const R* n, R wq, R k, cpx<R>& ds, cpx<R>& dd) {
  R d0 = y[0] - x[0], d1 = y[1] - x[1], d2 = y[2] - x[2];
  R r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
  R sn, cs;
  gsc(k * r, &sn, &cs);
  R c = wq / R(4.0 * BEM_PI);
  // i e^{ikr} = -sin + i cos
  ds.re += c * (-sn);
  ds.im += c * cs;
  R dn = d0 * n[0] + d1 * n[1] + d2 * n[2];
  R f = -c * k * dn / r;
  dd.re += f * cs;
  dd.im += f * sn;
}

template <typename R>
struct GTriT {
  R v[3][3], n[3], c[3], area, h;
};
typedef GTriT<double> GTri;

__device__ void gload(const double* __restrict__ qpt, const double* __restrict__ nrm, const double* __restrict__ cent,
                      const double* __restrict__ area, const double* __restrict__ hmax, int j, GTri& t) {
  for (int d = 0; d < 3; ++d) {
    t.c[d] = cent[3 * j + d];
    t.n[d] = nrm[3 * j + d];
    for (int a = 0; a < 3; ++a) t.v[a][d] = 2.0 * qpt[9 * j + 3 * a + d] - t.c[d];
  }
  t.area = area[j];
  t.h = hmax[j];
}

// d/dk of rule R_L on triangle t (4^L congruent pieces, 3-point rule each)
template <typename R>
__device__ void dk_rule(const R* x, const GTriT<R>& t, int L, R k, cpx<R>& ds, cpx<R>& dd) {
  int npieces = 1 << (2 * L);
  R w = t.area / (R(3) * npieces);
  for (int piece = 0; piece < npieces; ++piece) {
    R a[3], b[3], c[3];
    for (int d = 0; d < 3; ++d) {
      a[d] = t.v[0][d];
      b[d] = t.v[1][d];
      c[d] = t.v[2][d];
    }
    int code = piece;
    for (int lvl = 0; lvl < L; ++lvl) {
      int child = code & 3;
      code >>= 2;
      R ab[3], bc[3], ca[3];
      for (int d = 0; d < 3; ++d) {
        ab[d] = R(0.5) * (a[d] + b[d]);
        bc[d] = R(0.5) * (b[d] + c[d]);
        ca[d] = R(0.5) * (c[d] + a[d]);
      }
      for (int d = 0; d < 3; ++d) {
        if (child == 0) {
          b[d] = ab[d];
          c[d] = ca[d];
        } else if (child == 1) {
          a[d] = ab[d];
          c[d] = bc[d];
        } else if (child == 2) {
          a[d] = ca[d];
          b[d] = bc[d];
        } else {
          a[d] = ab[d];
          b[d] = bc[d];
          c[d] = ca[d];
        }
      }
    }
    const R b0 = R(2) / R(3), b1 = R(1) / R(6);
    for (int q = 0; q < 3; ++q) {
      R y[3];
      for (int d = 0; d < 3; ++d)
        y[d] = (q == 0 ? b0 : b1) * a[d] + (q == 1 ? b0 : b1) * b[d] + (q == 2 ? b0 : b1) * c[d];
      dk_point(x, y, t.n, w, k, ds, dd);
    }
  }
}

// int_0^1 s e^{i a s} ds  (series for small a, closed form otherwise)
__device__ zd moment1(double a) {
  if (fabs(a) < 0.5) {
    // sum_n (i a)^n / (n! (n + 2))
    zd acc = cmk(0.0, 0.0), term = cmk(1.0, 0.0);  // (i a)^n / n!
#pragma unroll
    for (int n = 0; n < 30; ++n) {  // unrolled: the reciprocals fold to constants
      acc = acc + (1.0 / (n + 2.0)) * term;
      term = (1.0 / (n + 1.0)) * (term * cmk(0.0, a));
    }
    return acc;
  }
  double sn, cs;
  sincos(a, &sn, &cs);
  zd e = cmk(cs, sn);
  // e/(ia) + (e - 1)/a^2
  zd t1 = (1.0 / a) * (e * cmk(0.0, -1.0));
  zd t2 = (1.0 / (a * a)) * (e - cmk(1.0, 0.0));
  return t1 + t2;
}

__constant__ double c_ggl_x[32];
__constant__ double c_ggl_w[32];

// dS_ii/dk = (1/4 pi) sum_edges int (int_0^rho i t e^{ikt} dt) dphi, with
// tan(phi) = sinh(u): rho = d cosh(u), dphi = du / cosh(u)
__device__ zd dk_self(const GTri& t, double k, int lane) {
  // the 32 Gauss-Legendre points of each edge split over the lanes of a warp;
  // every lane returns the warp's sum
  zd acc = cmk(0.0, 0.0);
  const double xq = c_ggl_x[lane], wgl = c_ggl_w[lane];
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
    double u0 = asinh(-pr / dist), u1 = asinh((len - pr) / dist);
    double half = 0.5 * (u1 - u0), mid = 0.5 * (u1 + u0);
    const double u = mid + half * xq;
    const double eu = exp(u), ch = 0.5 * (eu + 1.0 / eu), ich = 1.0 / ch;
    const double rho = dist * ch;
    const zd m = moment1(k * rho);                       // int_0^1 s e^{i k rho s} ds
    const zd inner = (rho * rho) * (cmk(0.0, 1.0) * m);  // i rho^2 m
    acc = acc + (half * wgl * ich) * inner;
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
    acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
  }
  return (1.0 / (4.0 * BEM_PI)) * acc;
}

// corrections: (d/dk of the refined / exact entry) - (d/dk of R_0) for every
// correction pair; FP64, except the non-self pairs of the mixed modes (f32),
// which run in FP32 relative to the target
__global__ void k_grad_k_corr(int64_t nt, int nrhs, int f32, double k, const double* __restrict__ cent,
                              const double* __restrict__ qpt, const double* __restrict__ nrm,
                              const double* __restrict__ area, const double* __restrict__ hmax,
                              const int* __restrict__ ptr, const int* __restrict__ col, const double4* __restrict__ yx,
                              const double2* __restrict__ gs, double* out) {
  int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  double part = 0.0;
  if (i < nt) {
    double x[3] = {cent[3 * i], cent[3 * i + 1], cent[3 * i + 2]};
    for (int e = ptr[i] + lane; e < ptr[i + 1]; e += 32) {
      int j = col[e];
      if ((int64_t)j == i) continue;  // the self pair: k_grad_k_self
      GTri t;
      gload(qpt, nrm, cent, area, hmax, j, t);
      zd s0 = cmk(0.0, 0.0), d0 = cmk(0.0, 0.0), s1 = cmk(0.0, 0.0), d1 = cmk(0.0, 0.0);
      if (f32 && (int64_t)j != i) {
        // mixed modes: both rules of a non-self pair in FP32, relative to the target
        double dd3[3] = {t.c[0] - x[0], t.c[1] - x[1], t.c[2] - x[2]};
        double dist = sqrt(dd3[0] * dd3[0] + dd3[1] * dd3[1] + dd3[2] * dd3[2]);
        int L = dist < 2.0 * t.h ? 2 : (dist < 4.0 * t.h ? 1 : 0);
        if (L == 0) continue;
        GTriT<float> tf;
        for (int a = 0; a < 3; ++a)
          for (int d = 0; d < 3; ++d) tf.v[a][d] = (float)(t.v[a][d] - x[d]);
        for (int d = 0; d < 3; ++d) {
          tf.n[d] = (float)t.n[d];
          tf.c[d] = (float)(t.c[d] - x[d]);
        }
        tf.area = (float)t.area;
        tf.h = (float)t.h;
        const float x0[3] = {0.f, 0.f, 0.f};
        cpx<float> s0f = cmk(0.f, 0.f), d0f = s0f, s1f = s0f, d1f = s0f;
        dk_rule(x0, tf, 0, (float)k, s0f, d0f);
        dk_rule(x0, tf, L, (float)k, s1f, d1f);
        const zd csf = cmk((double)(s1f.re - s0f.re), (double)(s1f.im - s0f.im));
        const zd cdf = cmk((double)(d1f.re - d0f.re), (double)(d1f.im - d0f.im));
        for (int r = 0; r < nrhs; ++r) {
          double4 uy = yx[(int64_t)r * nt + j];
          zd v = csf * cmk(uy.x, uy.y) - cdf * cmk(uy.z, uy.w);
          double2 g = gs[(int64_t)r * nt + i];
          part += g.x * v.re + g.y * v.im;
        }
        continue;
      }
      dk_rule(x, t, 0, k, s0, d0);
      {
        double dd[3] = {t.c[0] - x[0], t.c[1] - x[1], t.c[2] - x[2]};
        double dist = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
        int L = dist < 2.0 * t.h ? 2 : (dist < 4.0 * t.h ? 1 : 0);
        if (L == 0) {
          s1 = s0;
          d1 = d0;
        } else {
          dk_rule(x, t, L, k, s1, d1);
        }
      }
      zd cs = s1 - s0, cd = d1 - d0;
      for (int r = 0; r < nrhs; ++r) {
        double4 uy = yx[(int64_t)r * nt + j];
        zd v = cs * cmk(uy.x, uy.y) - cd * cmk(uy.z, uy.w);
        double2 g = gs[(int64_t)r * nt + i];
        part += g.x * v.re + g.y * v.im;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if (lane == 0 && part != 0.0) atomicAdd(out, part);
}

// the self pairs: (d/dk of the exact S_ii) - (d/dk of R_0 at the own centroid),
// one element per thread (their FP64 loops run side by side)
__global__ void k_grad_k_self(int64_t nt, int nrhs, double k, const double* __restrict__ cent,
                              const double* __restrict__ qpt, const double* __restrict__ nrm,
                              const double* __restrict__ area, const double* __restrict__ hmax,
                              const double4* __restrict__ yx, const double2* __restrict__ gs, double* out) {
  // one warp per element (the lanes split the exact term's quadrature)
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  double part = 0.0;
  if (i < nt) {
    GTri t;
    gload(qpt, nrm, cent, area, hmax, (int)i, t);
    const zd se = dk_self(t, k, lane);
    if (lane == 0) {
      const double x[3] = {t.c[0], t.c[1], t.c[2]};
      zd s0 = cmk(0.0, 0.0), d0 = cmk(0.0, 0.0);
      dk_rule(x, t, 0, k, s0, d0);
      const zd cs = se - s0, cd = cmk(0.0, 0.0) - d0;
      for (int r = 0; r < nrhs; ++r) {
        const double4 uy = yx[(int64_t)r * nt + i];
        const zd v = cs * cmk(uy.x, uy.y) - cd * cmk(uy.z, uy.w);
        const double2 g = gs[(int64_t)r * nt + i];
        part += g.x * v.re + g.y * v.im;
      }
    }
  }
  // one atomic add per block of four elements
  __shared__ double s_part[4];
  if (lane == 0) s_part[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    const double sum = s_part[0] + s_part[1] + s_part[2] + s_part[3];
    if (sum != 0.0) atomicAdd(out, sum);
  }
}

void bem_gl_host(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(BEM_PI * (i + 0.75) / (n + 0.5));
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
      if (fabs(dz) < 1e-16) {
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

extern "C" int bem_grad(bem_handle* h, int nrhs, int dtype, const void* g, const void* x, const void* y,
                        double* dvertices, double* dk, void* stream) {
  bem_set_error("");
  if (!h) return bem_fail(BEM_ERR_INVALID_ARG, "handle is NULL");
  if (nrhs < 1 || nrhs > h->nrhs_max) return bem_fail(BEM_ERR_INVALID_ARG, "nrhs out of [1, max_nrhs]");
  if (dtype != BEM_C64 && dtype != BEM_C128) return bem_fail(BEM_ERR_INVALID_ARG, "dtype must be BEM_C64 or BEM_C128");
  if (!g || (!x && !y)) return bem_fail(BEM_ERR_INVALID_ARG, "g and at least one of x, y are required");
  if (!dk && !dvertices) return bem_fail(BEM_ERR_INVALID_ARG, "dk and dvertices are both NULL");
  cudaPointerAttributes pa;
  if (dvertices && (cudaPointerGetAttributes(&pa, dvertices) != cudaSuccess || pa.type == cudaMemoryTypeDevice)) {
    cudaGetLastError();
    return bem_fail(BEM_ERR_INVALID_ARG, "dvertices must be a host pointer");
  }
  cudaStream_t s = (cudaStream_t)stream;
  int64_t nt = h->nt;
  double4* yx;
  double2* gs;
  double* acc;
  // scratch for this call (gradients are not on the matvec path)
  BEM_CUDA(cudaMallocAsync((void**)&yx, sizeof(double4) * nt * nrhs, s));
  BEM_CUDA(cudaMallocAsync((void**)&gs, sizeof(double2) * nt * nrhs, s));
  BEM_CUDA(cudaMallocAsync((void**)&acc, sizeof(double), s));
  BEM_CUDA(cudaMemsetAsync(acc, 0, sizeof(double), s));
  if (dtype == BEM_C128)
    k_grad_prologue<double><<<nblk(nt, 256), 256, 0, s>>>(nt, nrhs, h->perm, (const double*)g, (const double*)x,
                                                          (const double*)y, yx, gs);
  else
    k_grad_prologue<float><<<nblk(nt, 256), 256, 0, s>>>(nt, nrhs, h->perm, (const float*)g, (const float*)x,
                                                         (const float*)y, yx, gs);
  BEM_CUDA(cudaGetLastError());
  // the regular rule (vertex terms, and dL/dk's regular part); with the
  // vertices asked for, the correction and self kernels of the vertex
  // gradient add dL/dk's corrections on the same quadrature points too
  BEM_TRY(bem_grad_vertices(h, nrhs, yx, gs, dvertices, dk ? acc : nullptr, s));
  if (!dk || dvertices) {
    if (dk) BEM_CUDA(cudaMemcpyAsync(dk, acc, sizeof(double), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaFreeAsync(yx, s));
    BEM_CUDA(cudaFreeAsync(gs, s));
    BEM_CUDA(cudaFreeAsync(acc, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    return bem_check_device_error(h, s);
  }
  double glx[32], glw[32];
  bem_gl_host(32, glx, glw);
  BEM_CUDA(cudaMemcpyToSymbolAsync(c_ggl_x, glx, sizeof(glx), 0, cudaMemcpyHostToDevice, s));
  BEM_CUDA(cudaMemcpyToSymbolAsync(c_ggl_w, glw, sizeof(glw), 0, cudaMemcpyHostToDevice, s));
  k_grad_k_corr<<<nblk(nt * 32, 128), 128, 0, s>>>(nt, nrhs, bem_is_fp64(h) ? 0 : 1, h->k, h->cent, h->qpt, h->nrm, h->area, h->hmax,
                                                   h->corr_ptr, h->corr_col, yx, gs, acc);
  BEM_CUDA(cudaGetLastError());
  k_grad_k_self<<<nblk(nt * 32, 128), 128, 0, s>>>(nt, nrhs, h->k, h->cent, h->qpt, h->nrm, h->area, h->hmax, yx, gs,
                                               acc);
  BEM_CUDA(cudaGetLastError());
  BEM_CUDA(cudaMemcpyAsync(dk, acc, sizeof(double), cudaMemcpyDeviceToHost, s));
  BEM_CUDA(cudaFreeAsync(yx, s));
  BEM_CUDA(cudaFreeAsync(gs, s));
  BEM_CUDA(cudaFreeAsync(acc, s));
  BEM_CUDA(cudaStreamSynchronize(s));
  return BEM_OK;
}
