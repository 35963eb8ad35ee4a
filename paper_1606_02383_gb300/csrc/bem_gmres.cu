// bem_gmres.cu -- restarted GMRES for (1/2 I - D) x = b (Section 2.3, Eq. (GMRES)
// without the FEM coupling term; Section 3: GMRES with a relative tolerance).
//
// All right-hand sides run in lockstep so every iteration makes one multi-rhs
// operator apply.  Krylov vectors, dot products and updates are FP64 on the
// device; orthogonalisation is classical Gram-Schmidt applied twice (CGS2).
// The small Hessenberg least-squares problem (Givens rotations) is solved on
// the host, which reads j+2 coefficients per rhs after every iteration.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "bem_common.cuh"

typedef std::complex<double> hz;
static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

#define GM_CHUNKS 128

// partial[(r*(nv) + i)*GM_CHUNKS + chunk] = sum over the chunk of conj(V_i[r]) w[r]
__global__ void k_gm_dots(int64_t n, int nv, int nrhs, const double* __restrict__ V, int64_t vstride,
                          const double* __restrict__ w, double* partial) {
  int chunk = blockIdx.x, i = blockIdx.y, r = blockIdx.z;
  int64_t per = (n + GM_CHUNKS - 1) / GM_CHUNKS;
  int64_t a = chunk * per, b = min(n, a + per);
  const double* v = V + i * vstride + 2 * (int64_t)r * n;
  const double* ww = w + 2 * (int64_t)r * n;
  double sre = 0.0, sim = 0.0;
  for (int64_t e = a + threadIdx.x; e < b; e += blockDim.x) {
    double vr = v[2 * e], vi = v[2 * e + 1], wr = ww[2 * e], wi = ww[2 * e + 1];
    sre += vr * wr + vi * wi;
    sim += vr * wi - vi * wr;
  }
  __shared__ double sh[2][256];
  sh[0][threadIdx.x] = sre;
  sh[1][threadIdx.x] = sim;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + st];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int64_t o = ((int64_t)r * nv + i) * GM_CHUNKS + chunk;
    partial[2 * o] = sh[0][0];
    partial[2 * o + 1] = sh[1][0];
  }
}

// out[r*nv + i] (+)= sum over chunks
__global__ void k_gm_reduce(int nv, int nrhs, const double* __restrict__ partial, double* out, int accumulate) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nv * nrhs) return;
  double sre = 0.0, sim = 0.0;
  for (int c = 0; c < GM_CHUNKS; ++c) {
    sre += partial[2 * ((int64_t)t * GM_CHUNKS + c)];
    sim += partial[2 * ((int64_t)t * GM_CHUNKS + c) + 1];
  }
  if (accumulate) {
    out[2 * t] += sre;
    out[2 * t + 1] += sim;
  } else {
    out[2 * t] = sre;
    out[2 * t + 1] = sim;
  }
}

// w[r] -= sum_i coef[r*nv + i] V_i[r]   (coef from the latest dot round)
__global__ void k_gm_orth(int64_t n, int nv, int nrhs, const double* __restrict__ V, int64_t vstride,
                          const double* __restrict__ coef, double* w) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (e >= n) return;
  double wr = w[2 * ((int64_t)r * n + e)], wi = w[2 * ((int64_t)r * n + e) + 1];
  for (int i = 0; i < nv; ++i) {
    double cr = coef[2 * (r * nv + i)], ci = coef[2 * (r * nv + i) + 1];
    const double* v = V + i * vstride + 2 * ((int64_t)r * n + e);
    wr -= cr * v[0] - ci * v[1];
    wi -= cr * v[1] + ci * v[0];
  }
  w[2 * ((int64_t)r * n + e)] = wr;
  w[2 * ((int64_t)r * n + e) + 1] = wi;
}

// dst[r] = src[r] * scale[r] (complex src, real scale)
__global__ void k_gm_scale(int64_t n, const double* __restrict__ src, const double* __restrict__ scale, double* dst) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (e >= n) return;
  double s = scale[r];
  dst[2 * ((int64_t)r * n + e)] = src[2 * ((int64_t)r * n + e)] * s;
  dst[2 * ((int64_t)r * n + e) + 1] = src[2 * ((int64_t)r * n + e) + 1] * s;
}

// x[r] += sum_i y[r][i] V_i[r]
__global__ void k_gm_update_x(int64_t n, int nv, const double* __restrict__ V, int64_t vstride,
                              const double* __restrict__ y, double* x) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (e >= n) return;
  double xr = x[2 * ((int64_t)r * n + e)], xi = x[2 * ((int64_t)r * n + e) + 1];
  for (int i = 0; i < nv; ++i) {
    double yr = y[2 * (r * nv + i)], yi = y[2 * (r * nv + i) + 1];
    const double* v = V + i * vstride + 2 * ((int64_t)r * n + e);
    xr += yr * v[0] - yi * v[1];
    xi += yr * v[1] + yi * v[0];
  }
  x[2 * ((int64_t)r * n + e)] = xr;
  x[2 * ((int64_t)r * n + e) + 1] = xi;
}

// r = b - z  (all complex double)
__global__ void k_gm_sub(int64_t m, const double* __restrict__ b, const double* __restrict__ z, double* r) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m) return;
  r[e] = b[e] - z[e];
}

__global__ void k_c64_to_c128(int64_t m, const float* __restrict__ a, double* b) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < m) b[e] = (double)a[e];
}
__global__ void k_c128_to_c64(int64_t m, const double* __restrict__ a, float* b) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < m) b[e] = (float)a[e];
}

struct Gm {
  bem_handle* h;
  int nrhs;
  int64_t n;
  cudaStream_t s;
  double *V, *w, *partial, *coef, *coef2, *nrm, *scale, *y, *tmp;
  int64_t vstride;
};

static int gm_apply(Gm& g, const double* in, double* out) {
  BEM_TRY(bem_prologue(g.h, g.nrhs, BEM_C128, in, nullptr, g.s));
  BEM_TRY(bem_apply_sorted(g.h, g.nrhs, g.s));
  BEM_TRY(bem_epilogue(g.h, g.nrhs, BEM_C128, in, out, 1, g.s));
  return BEM_OK;
}

// squared norms of the nrhs vectors in `w` into host array
static int gm_norms(Gm& g, const double* w, std::vector<double>& out) {
  dim3 grid(GM_CHUNKS, 1, g.nrhs);
  k_gm_dots<<<grid, 256, 0, g.s>>>(g.n, 1, g.nrhs, w, 0, w, g.partial);
  k_gm_reduce<<<nblk(g.nrhs, 128), 128, 0, g.s>>>(1, g.nrhs, g.partial, g.nrm, 0);
  std::vector<double> t(2 * g.nrhs);
  BEM_CUDA(cudaMemcpyAsync(t.data(), g.nrm, 2 * g.nrhs * sizeof(double), cudaMemcpyDeviceToHost, g.s));
  BEM_CUDA(cudaStreamSynchronize(g.s));
  out.resize(g.nrhs);
  for (int r = 0; r < g.nrhs; ++r) out[r] = std::sqrt(std::max(0.0, t[2 * r]));
  return BEM_OK;
}

int bem_gmres(bem_handle* h, int nrhs, int dtype, const void* b_in, void* x_out, double tol, int max_iter,
              int restart, int flags, int* iters_out, double* relres_out, cudaStream_t s) {
  int64_t n = h->nt;
  int m = std::min(restart, max_iter);
  Gm g;
  g.h = h;
  g.nrhs = nrhs;
  g.n = n;
  g.s = s;
  // workspace (re)allocation
  if (!h->gm_V || h->gm_restart < m || h->gm_nrhs < nrhs) {
    BEM_TRY(bem_alloc(h, &h->gm_V, (size_t)(m + 1) * nrhs * n * 2));
    BEM_TRY(bem_alloc(h, &h->gm_w, (size_t)nrhs * n * 2 * 3));
    BEM_TRY(bem_alloc(h, &h->gm_dots, (size_t)nrhs * (m + 1) * GM_CHUNKS * 2 + 4 * (size_t)nrhs * (m + 1) * 2 + 2 * nrhs));
    h->gm_restart = m;
    h->gm_nrhs = nrhs;
  }
  g.vstride = (int64_t)nrhs * n * 2;
  g.V = h->gm_V;
  g.w = h->gm_w;
  double* bb = h->gm_w + (size_t)nrhs * n * 2;      // b in C128
  double* xx = bb + (size_t)nrhs * n * 2;           // x in C128
  g.partial = h->gm_dots;
  g.coef = g.partial + (size_t)nrhs * (m + 1) * GM_CHUNKS * 2;
  g.coef2 = g.coef + (size_t)nrhs * (m + 1) * 2;
  g.y = g.coef2 + (size_t)nrhs * (m + 1) * 2;
  g.nrm = g.y + (size_t)nrhs * (m + 1) * 2;
  g.scale = g.nrm + (size_t)nrhs * (m + 1) * 2;
  int64_t tot = 2 * (int64_t)nrhs * n;
  if (dtype == BEM_C128) {
    BEM_CUDA(cudaMemcpyAsync(bb, b_in, tot * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (flags & BEM_GMRES_USE_X0) BEM_CUDA(cudaMemcpyAsync(xx, x_out, tot * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else {
    k_c64_to_c128<<<nblk(tot, 256), 256, 0, s>>>(tot, (const float*)b_in, bb);
    if (flags & BEM_GMRES_USE_X0) k_c64_to_c128<<<nblk(tot, 256), 256, 0, s>>>(tot, (const float*)x_out, xx);
  }
  if (!(flags & BEM_GMRES_USE_X0)) BEM_CUDA(cudaMemsetAsync(xx, 0, tot * sizeof(double), s));

  std::vector<double> bnorm;
  BEM_TRY(gm_norms(g, bb, bnorm));
  std::vector<double> relres(nrhs, 1.0);
  int it_total = 0;
  bool all_conv = false;
  dim3 gvec(nblk(n, 256), nrhs);
  while (it_total < max_iter && !all_conv) {
    // r0 = b - A x
    BEM_TRY(gm_apply(g, xx, g.w));
    k_gm_sub<<<nblk(tot, 256), 256, 0, s>>>(tot, bb, g.w, g.w);
    std::vector<double> beta;
    BEM_TRY(gm_norms(g, g.w, beta));
    std::vector<double> sc(nrhs);
    std::vector<bool> active(nrhs);
    all_conv = true;
    for (int r = 0; r < nrhs; ++r) {
      double bn = bnorm[r] > 0 ? bnorm[r] : 1.0;
      relres[r] = beta[r] / bn;
      active[r] = relres[r] > tol && beta[r] > 0.0;
      if (active[r]) all_conv = false;
      sc[r] = active[r] ? 1.0 / beta[r] : 0.0;
    }
    if (all_conv) break;
    BEM_CUDA(cudaMemcpyAsync(g.scale, sc.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
    k_gm_scale<<<gvec, 256, 0, s>>>(n, g.w, g.scale, g.V);
    // per-rhs small problem
    std::vector<std::vector<hz>> H(nrhs, std::vector<hz>((size_t)(m + 1) * m, 0.0));
    std::vector<std::vector<double>> cs(nrhs, std::vector<double>(m, 0.0));
    std::vector<std::vector<hz>> sn(nrhs, std::vector<hz>(m, 0.0));
    std::vector<std::vector<hz>> gg(nrhs, std::vector<hz>(m + 1, 0.0));
    std::vector<int> ncols(nrhs, 0);
    for (int r = 0; r < nrhs; ++r) gg[r][0] = beta[r];
    int j = 0;
    for (; j < m && it_total < max_iter; ++j) {
      double* vj = g.V + j * g.vstride;
      BEM_TRY(gm_apply(g, vj, g.w));
      int nv = j + 1;
      // CGS2
      dim3 gd(GM_CHUNKS, nv, nrhs);
      k_gm_dots<<<gd, 256, 0, s>>>(n, nv, nrhs, g.V, g.vstride, g.w, g.partial);
      k_gm_reduce<<<nblk(nv * nrhs, 128), 128, 0, s>>>(nv, nrhs, g.partial, g.coef, 0);
      k_gm_orth<<<gvec, 256, 0, s>>>(n, nv, nrhs, g.V, g.vstride, g.coef, g.w);
      k_gm_dots<<<gd, 256, 0, s>>>(n, nv, nrhs, g.V, g.vstride, g.w, g.partial);
      k_gm_reduce<<<nblk(nv * nrhs, 128), 128, 0, s>>>(nv, nrhs, g.partial, g.coef2, 0);
      k_gm_orth<<<gvec, 256, 0, s>>>(n, nv, nrhs, g.V, g.vstride, g.coef2, g.w);
      BEM_CUDA(cudaGetLastError());
      std::vector<double> hc(2 * nv * nrhs), hc2(2 * nv * nrhs);
      BEM_CUDA(cudaMemcpyAsync(hc.data(), g.coef, hc.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
      BEM_CUDA(cudaMemcpyAsync(hc2.data(), g.coef2, hc2.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
      std::vector<double> wn;
      BEM_TRY(gm_norms(g, g.w, wn));  // synchronises
      ++it_total;
      bool any = false;
      for (int r = 0; r < nrhs; ++r) {
        if (!active[r]) {
          sc[r] = 0.0;
          continue;
        }
        std::vector<hz>& Hr = H[r];
        for (int i = 0; i < nv; ++i)
          Hr[(size_t)i * m + j] = hz(hc[2 * (r * nv + i)] + hc2[2 * (r * nv + i)],
                                     hc[2 * (r * nv + i) + 1] + hc2[2 * (r * nv + i) + 1]);
        double hn = wn[r];
        Hr[(size_t)(j + 1) * m + j] = hn;
        for (int i = 0; i < j; ++i) {  // previous rotations
          hz a = Hr[(size_t)i * m + j], bq = Hr[(size_t)(i + 1) * m + j];
          Hr[(size_t)i * m + j] = cs[r][i] * a + sn[r][i] * bq;
          Hr[(size_t)(i + 1) * m + j] = -std::conj(sn[r][i]) * a + cs[r][i] * bq;
        }
        hz a = Hr[(size_t)j * m + j];
        double bq = std::abs(Hr[(size_t)(j + 1) * m + j]);
        double rho = std::hypot(std::abs(a), bq);
        if (std::abs(a) == 0.0) {
          cs[r][j] = 0.0;
          sn[r][j] = 1.0;
        } else {
          cs[r][j] = std::abs(a) / rho;
          sn[r][j] = (a / std::abs(a)) * bq / rho;
        }
        Hr[(size_t)j * m + j] = cs[r][j] * a + sn[r][j] * bq;
        Hr[(size_t)(j + 1) * m + j] = 0.0;
        gg[r][j + 1] = -std::conj(sn[r][j]) * gg[r][j];
        gg[r][j] = cs[r][j] * gg[r][j];
        ncols[r] = j + 1;
        double bn = bnorm[r] > 0 ? bnorm[r] : 1.0;
        relres[r] = std::abs(gg[r][j + 1]) / bn;
        bool breakdown = !(hn > 1e-14 * std::abs(Hr[(size_t)j * m + j]));
        if (relres[r] <= tol || breakdown) {
          active[r] = false;
          sc[r] = 0.0;
        } else {
          sc[r] = 1.0 / hn;
          any = true;
        }
      }
      if (!any) {
        ++j;
        break;
      }
      BEM_CUDA(cudaMemcpyAsync(g.scale, sc.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
      k_gm_scale<<<gvec, 256, 0, s>>>(n, g.w, g.scale, g.V + (j + 1) * g.vstride);
    }
    // solve the triangular systems and update x
    int nvmax = 0;
    for (int r = 0; r < nrhs; ++r) nvmax = std::max(nvmax, ncols[r]);
    if (nvmax > 0) {
      std::vector<double> yv(2 * (size_t)nrhs * nvmax, 0.0);
      for (int r = 0; r < nrhs; ++r) {
        int k = ncols[r];
        std::vector<hz> yy(k);
        for (int i = k - 1; i >= 0; --i) {
          hz acc = gg[r][i];
          for (int q = i + 1; q < k; ++q) acc -= H[r][(size_t)i * m + q] * yy[q];
          yy[i] = acc / H[r][(size_t)i * m + i];
        }
        for (int i = 0; i < k; ++i) {
          yv[2 * (r * nvmax + i)] = yy[i].real();
          yv[2 * (r * nvmax + i) + 1] = yy[i].imag();
        }
      }
      BEM_CUDA(cudaMemcpyAsync(g.y, yv.data(), yv.size() * sizeof(double), cudaMemcpyHostToDevice, s));
      k_gm_update_x<<<gvec, 256, 0, s>>>(n, nvmax, g.V, g.vstride, g.y, xx);
      BEM_CUDA(cudaGetLastError());
      BEM_CUDA(cudaStreamSynchronize(s));
    }
    all_conv = true;
    for (int r = 0; r < nrhs; ++r)
      if (relres[r] > tol) all_conv = false;
  }
  if (dtype == BEM_C128)
    BEM_CUDA(cudaMemcpyAsync(x_out, xx, tot * sizeof(double), cudaMemcpyDeviceToDevice, s));
  else
    k_c128_to_c64<<<nblk(tot, 256), 256, 0, s>>>(tot, xx, (float*)x_out);
  BEM_CUDA(cudaStreamSynchronize(s));
  if (iters_out) *iters_out = it_total;
  if (relres_out)
    for (int r = 0; r < nrhs; ++r) relres_out[r] = relres[r];
  for (int r = 0; r < nrhs; ++r)
    if (!(relres[r] <= tol)) return bem_fail(BEM_ERR_NOT_CONVERGED, "GMRES reached max_iter before tol");
  return BEM_OK;
}
