// bem_gmres.cu -- restarted GMRES for (1/2 I - D) x = b (Section 2.3, Eq. (GMRES)
// without the FEM coupling term; Section 3: GMRES with a relative tolerance).
//
// The core solves `ncol` independent systems in lockstep: column c is the
// complex segment [off[c], off[c] + len[c]) of one block vector of length M,
// and every iteration makes one apply of the whole block (a multi-rhs apply of
// one operator, or one batch apply of many operators).  Krylov vectors, dot
// products and updates are FP64 on the device; orthogonalisation is classical
// Gram-Schmidt applied twice (CGS2).  The small Hessenberg least-squares
// problem (Givens rotations) of every column is solved on the host, which reads
// j+2 coefficients per column after every iteration.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "bem_common.cuh"

typedef std::complex<double> hz;
static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

#define GM_CHUNKS 128

// colof[off[c] + e] = c for every element of every column
__global__ void k_gm_colof(const int64_t* __restrict__ off, const int64_t* __restrict__ len, int* colof) {
  const int c = blockIdx.y;
  const int64_t n = len[c], o = off[c];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    colof[o + e] = c;
}

// partial[(c*nv + i)*GM_CHUNKS + chunk] = sum over the chunk of conj(V_i[c]) w[c]
__global__ void k_gm_dots(int nv, const int64_t* __restrict__ off, const int64_t* __restrict__ len,
                          const double* __restrict__ V, int64_t vstride, const double* __restrict__ w,
                          double* partial) {
  int chunk = blockIdx.x, i = blockIdx.y, c = blockIdx.z;
  const int64_t n = len[c];
  int64_t per = (n + GM_CHUNKS - 1) / GM_CHUNKS;
  int64_t a = chunk * per, b = min(n, a + per);
  const double* v = V + i * vstride + 2 * off[c];
  const double* ww = w + 2 * off[c];
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
    int64_t o = ((int64_t)c * nv + i) * GM_CHUNKS + chunk;
    partial[2 * o] = sh[0][0];
    partial[2 * o + 1] = sh[1][0];
  }
}

// out[c*nv + i] = sum over chunks
__global__ void k_gm_reduce(int nv, int ncol, const double* __restrict__ partial, double* out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nv * ncol) return;
  double sre = 0.0, sim = 0.0;
  for (int c = 0; c < GM_CHUNKS; ++c) {
    sre += partial[2 * ((int64_t)t * GM_CHUNKS + c)];
    sim += partial[2 * ((int64_t)t * GM_CHUNKS + c) + 1];
  }
  out[2 * t] = sre;
  out[2 * t + 1] = sim;
}

// w -= sum_i coef[c*nv + i] V_i   on every element e of column c = colof[e]
__global__ void k_gm_orth(int64_t M, int nv, const int* __restrict__ colof, const double* __restrict__ V,
                          int64_t vstride, const double* __restrict__ coef, double* w) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= M) return;
  const int c = colof[e];
  double wr = w[2 * e], wi = w[2 * e + 1];
  for (int i = 0; i < nv; ++i) {
    double cr = coef[2 * (c * nv + i)], ci = coef[2 * (c * nv + i) + 1];
    const double* v = V + i * vstride + 2 * e;
    wr -= cr * v[0] - ci * v[1];
    wi -= cr * v[1] + ci * v[0];
  }
  w[2 * e] = wr;
  w[2 * e + 1] = wi;
}

// dst = src * scale[column] (complex src, real scale)
__global__ void k_gm_scale(int64_t M, const int* __restrict__ colof, const double* __restrict__ src,
                           const double* __restrict__ scale, double* dst) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= M) return;
  double s = scale[colof[e]];
  dst[2 * e] = src[2 * e] * s;
  dst[2 * e + 1] = src[2 * e + 1] * s;
}

// x += sum_i y[c][i] V_i
__global__ void k_gm_update_x(int64_t M, int nv, const int* __restrict__ colof, const double* __restrict__ V,
                              int64_t vstride, const double* __restrict__ y, double* x) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= M) return;
  const int c = colof[e];
  double xr = x[2 * e], xi = x[2 * e + 1];
  for (int i = 0; i < nv; ++i) {
    double yr = y[2 * (c * nv + i)], yi = y[2 * (c * nv + i) + 1];
    const double* v = V + i * vstride + 2 * e;
    xr += yr * v[0] - yi * v[1];
    xi += yr * v[1] + yi * v[0];
  }
  x[2 * e] = xr;
  x[2 * e + 1] = xi;
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

namespace {

// stream-ordered scratch of one solve, released on every return path
struct GmScratch {
  cudaStream_t s;
  std::vector<void*> p;
  ~GmScratch() {
    for (void* q : p) cudaFreeAsync(q, s);
  }
  template <typename T>
  int get(T** out, size_t count) {
    void* q = nullptr;
    BEM_CUDA(cudaMallocAsync(&q, std::max<size_t>(count, 1) * sizeof(T), s));
    p.push_back(q);
    *out = (T*)q;
    return BEM_OK;
  }
};

struct GmCore {
  bem_gm_apply_fn apply;
  void* ctx;
  int ncol;
  int64_t M;
  cudaStream_t s;
  double *V, *w, *bb, *xx, *partial, *coef, *coef2, *y, *nrm, *scale;
  int64_t vstride;
  int64_t *d_off, *d_len;
  int* colof;
};

// norms of the ncol columns of `w` into a host array (synchronises)
int gm_norms(GmCore& g, const double* w, std::vector<double>& out) {
  dim3 grid(GM_CHUNKS, 1, g.ncol);
  k_gm_dots<<<grid, 256, 0, g.s>>>(1, g.d_off, g.d_len, w, 0, w, g.partial);
  k_gm_reduce<<<nblk(g.ncol, 128), 128, 0, g.s>>>(1, g.ncol, g.partial, g.nrm);
  std::vector<double> t(2 * (size_t)g.ncol);
  BEM_CUDA(cudaMemcpyAsync(t.data(), g.nrm, t.size() * sizeof(double), cudaMemcpyDeviceToHost, g.s));
  BEM_CUDA(cudaStreamSynchronize(g.s));
  out.resize(g.ncol);
  for (int c = 0; c < g.ncol; ++c) out[c] = std::sqrt(std::max(0.0, t[2 * c]));
  return BEM_OK;
}

}  // namespace

int bem_gmres_core(bem_gm_apply_fn apply, void* ctx, int ncol, int64_t M, const int64_t* off, const int64_t* len,
                   int dtype, const void* b_in, void* x_out, double tol, int max_iter, int restart, int flags,
                   int* iters_out, double* relres_out, cudaStream_t s) {
  const int m = std::max(1, std::min(restart, max_iter));
  GmScratch sc_{s, {}};
  GmCore g;
  g.apply = apply;
  g.ctx = ctx;
  g.ncol = ncol;
  g.M = M;
  g.s = s;
  g.vstride = 2 * M;
  BEM_TRY(sc_.get(&g.V, (size_t)(m + 1) * 2 * M));
  BEM_TRY(sc_.get(&g.w, 2 * (size_t)M));
  BEM_TRY(sc_.get(&g.bb, 2 * (size_t)M));
  BEM_TRY(sc_.get(&g.xx, 2 * (size_t)M));
  BEM_TRY(sc_.get(&g.partial, (size_t)ncol * (m + 1) * GM_CHUNKS * 2));
  BEM_TRY(sc_.get(&g.coef, (size_t)ncol * (m + 1) * 2));
  BEM_TRY(sc_.get(&g.coef2, (size_t)ncol * (m + 1) * 2));
  BEM_TRY(sc_.get(&g.y, (size_t)ncol * (m + 1) * 2));
  BEM_TRY(sc_.get(&g.nrm, (size_t)ncol * 2));
  BEM_TRY(sc_.get(&g.scale, (size_t)ncol));
  BEM_TRY(sc_.get(&g.d_off, (size_t)ncol));
  BEM_TRY(sc_.get(&g.d_len, (size_t)ncol));
  BEM_TRY(sc_.get(&g.colof, (size_t)M));
  BEM_CUDA(cudaMemcpyAsync(g.d_off, off, ncol * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  BEM_CUDA(cudaMemcpyAsync(g.d_len, len, ncol * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  k_gm_colof<<<dim3(64, ncol), 256, 0, s>>>(g.d_off, g.d_len, g.colof);
  const int64_t tot = 2 * M;
  if (dtype == BEM_C128) {
    BEM_CUDA(cudaMemcpyAsync(g.bb, b_in, tot * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (flags & BEM_GMRES_USE_X0)
      BEM_CUDA(cudaMemcpyAsync(g.xx, x_out, tot * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else {
    k_c64_to_c128<<<nblk(tot, 256), 256, 0, s>>>(tot, (const float*)b_in, g.bb);
    if (flags & BEM_GMRES_USE_X0) k_c64_to_c128<<<nblk(tot, 256), 256, 0, s>>>(tot, (const float*)x_out, g.xx);
  }
  if (!(flags & BEM_GMRES_USE_X0)) BEM_CUDA(cudaMemsetAsync(g.xx, 0, tot * sizeof(double), s));
  BEM_CUDA(cudaGetLastError());

  std::vector<double> bnorm;
  BEM_TRY(gm_norms(g, g.bb, bnorm));
  std::vector<double> relres(ncol, 1.0);
  int it_total = 0;
  bool all_conv = false;
  const unsigned gvec = nblk(M, 256);
  while (it_total < max_iter && !all_conv) {
    // r0 = b - A x
    BEM_TRY(g.apply(g.ctx, g.xx, g.w, s));
    k_gm_sub<<<nblk(tot, 256), 256, 0, s>>>(tot, g.bb, g.w, g.w);
    std::vector<double> beta;
    BEM_TRY(gm_norms(g, g.w, beta));
    std::vector<double> sc(ncol);
    std::vector<bool> active(ncol);
    all_conv = true;
    for (int c = 0; c < ncol; ++c) {
      double bn = bnorm[c] > 0 ? bnorm[c] : 1.0;
      relres[c] = beta[c] / bn;
      active[c] = relres[c] > tol && beta[c] > 0.0;
      if (active[c]) all_conv = false;
      sc[c] = active[c] ? 1.0 / beta[c] : 0.0;
    }
    if (all_conv) break;
    BEM_CUDA(cudaMemcpyAsync(g.scale, sc.data(), ncol * sizeof(double), cudaMemcpyHostToDevice, s));
    k_gm_scale<<<gvec, 256, 0, s>>>(M, g.colof, g.w, g.scale, g.V);
    // per-column small problem
    std::vector<std::vector<hz>> H(ncol, std::vector<hz>((size_t)(m + 1) * m, 0.0));
    std::vector<std::vector<double>> cs(ncol, std::vector<double>(m, 0.0));
    std::vector<std::vector<hz>> sn(ncol, std::vector<hz>(m, 0.0));
    std::vector<std::vector<hz>> gg(ncol, std::vector<hz>(m + 1, 0.0));
    std::vector<int> ncols(ncol, 0);
    for (int c = 0; c < ncol; ++c) gg[c][0] = beta[c];
    int j = 0;
    for (; j < m && it_total < max_iter; ++j) {
      double* vj = g.V + j * g.vstride;
      BEM_TRY(g.apply(g.ctx, vj, g.w, s));
      int nv = j + 1;
      // CGS2
      dim3 gd(GM_CHUNKS, nv, ncol);
      k_gm_dots<<<gd, 256, 0, s>>>(nv, g.d_off, g.d_len, g.V, g.vstride, g.w, g.partial);
      k_gm_reduce<<<nblk(nv * ncol, 128), 128, 0, s>>>(nv, ncol, g.partial, g.coef);
      k_gm_orth<<<gvec, 256, 0, s>>>(M, nv, g.colof, g.V, g.vstride, g.coef, g.w);
      k_gm_dots<<<gd, 256, 0, s>>>(nv, g.d_off, g.d_len, g.V, g.vstride, g.w, g.partial);
      k_gm_reduce<<<nblk(nv * ncol, 128), 128, 0, s>>>(nv, ncol, g.partial, g.coef2);
      k_gm_orth<<<gvec, 256, 0, s>>>(M, nv, g.colof, g.V, g.vstride, g.coef2, g.w);
      BEM_CUDA(cudaGetLastError());
      std::vector<double> hc(2 * (size_t)nv * ncol), hc2(2 * (size_t)nv * ncol);
      BEM_CUDA(cudaMemcpyAsync(hc.data(), g.coef, hc.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
      BEM_CUDA(cudaMemcpyAsync(hc2.data(), g.coef2, hc2.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
      std::vector<double> wn;
      BEM_TRY(gm_norms(g, g.w, wn));  // synchronises
      ++it_total;
      bool any = false;
      for (int c = 0; c < ncol; ++c) {
        if (!active[c]) {
          sc[c] = 0.0;
          continue;
        }
        std::vector<hz>& Hc = H[c];
        for (int i = 0; i < nv; ++i)
          Hc[(size_t)i * m + j] = hz(hc[2 * (c * nv + i)] + hc2[2 * (c * nv + i)],
                                     hc[2 * (c * nv + i) + 1] + hc2[2 * (c * nv + i) + 1]);
        double hn = wn[c];
        Hc[(size_t)(j + 1) * m + j] = hn;
        for (int i = 0; i < j; ++i) {  // previous rotations
          hz a = Hc[(size_t)i * m + j], bq = Hc[(size_t)(i + 1) * m + j];
          Hc[(size_t)i * m + j] = cs[c][i] * a + sn[c][i] * bq;
          Hc[(size_t)(i + 1) * m + j] = -std::conj(sn[c][i]) * a + cs[c][i] * bq;
        }
        hz a = Hc[(size_t)j * m + j];
        double bq = std::abs(Hc[(size_t)(j + 1) * m + j]);
        double rho = std::hypot(std::abs(a), bq);
        if (std::abs(a) == 0.0) {
          cs[c][j] = 0.0;
          sn[c][j] = 1.0;
        } else {
          cs[c][j] = std::abs(a) / rho;
          sn[c][j] = (a / std::abs(a)) * bq / rho;
        }
        Hc[(size_t)j * m + j] = cs[c][j] * a + sn[c][j] * bq;
        Hc[(size_t)(j + 1) * m + j] = 0.0;
        gg[c][j + 1] = -std::conj(sn[c][j]) * gg[c][j];
        gg[c][j] = cs[c][j] * gg[c][j];
        ncols[c] = j + 1;
        double bn = bnorm[c] > 0 ? bnorm[c] : 1.0;
        relres[c] = std::abs(gg[c][j + 1]) / bn;
        bool breakdown = !(hn > 1e-14 * std::abs(Hc[(size_t)j * m + j]));
        if (relres[c] <= tol || breakdown) {
          active[c] = false;
          sc[c] = 0.0;
        } else {
          sc[c] = 1.0 / hn;
          any = true;
        }
      }
      if (!any) {
        ++j;
        break;
      }
      BEM_CUDA(cudaMemcpyAsync(g.scale, sc.data(), ncol * sizeof(double), cudaMemcpyHostToDevice, s));
      k_gm_scale<<<gvec, 256, 0, s>>>(M, g.colof, g.w, g.scale, g.V + (j + 1) * g.vstride);
    }
    // solve the triangular systems and update x
    int nvmax = 0;
    for (int c = 0; c < ncol; ++c) nvmax = std::max(nvmax, ncols[c]);
    if (nvmax > 0) {
      std::vector<double> yv(2 * (size_t)ncol * nvmax, 0.0);
      for (int c = 0; c < ncol; ++c) {
        int k = ncols[c];
        std::vector<hz> yy(k);
        for (int i = k - 1; i >= 0; --i) {
          hz acc = gg[c][i];
          for (int q = i + 1; q < k; ++q) acc -= H[c][(size_t)i * m + q] * yy[q];
          yy[i] = acc / H[c][(size_t)i * m + i];
        }
        for (int i = 0; i < k; ++i) {
          yv[2 * (c * nvmax + i)] = yy[i].real();
          yv[2 * (c * nvmax + i) + 1] = yy[i].imag();
        }
      }
      BEM_CUDA(cudaMemcpyAsync(g.y, yv.data(), yv.size() * sizeof(double), cudaMemcpyHostToDevice, s));
      k_gm_update_x<<<gvec, 256, 0, s>>>(M, nvmax, g.colof, g.V, g.vstride, g.y, g.xx);
      BEM_CUDA(cudaGetLastError());
      BEM_CUDA(cudaStreamSynchronize(s));
    }
    all_conv = true;
    for (int c = 0; c < ncol; ++c)
      if (relres[c] > tol) all_conv = false;
  }
  if (dtype == BEM_C128)
    BEM_CUDA(cudaMemcpyAsync(x_out, g.xx, tot * sizeof(double), cudaMemcpyDeviceToDevice, s));
  else
    k_c128_to_c64<<<nblk(tot, 256), 256, 0, s>>>(tot, g.xx, (float*)x_out);
  BEM_CUDA(cudaStreamSynchronize(s));
  if (iters_out) *iters_out = it_total;
  if (relres_out)
    for (int c = 0; c < ncol; ++c) relres_out[c] = relres[c];
  for (int c = 0; c < ncol; ++c)
    if (!(relres[c] <= tol)) return bem_fail(BEM_ERR_NOT_CONVERGED, "GMRES reached max_iter before tol");
  return BEM_OK;
}

// ---------------------------------------------------------- one operator --
namespace {
struct OneOp {
  bem_handle* h;
  int nrhs;
};
int one_op_apply(void* ctx, const double* in, double* out, cudaStream_t s) {
  OneOp* o = (OneOp*)ctx;
  BEM_TRY(bem_prologue(o->h, o->nrhs, BEM_C128, in, nullptr, s));
  BEM_TRY(bem_apply_sorted(o->h, o->nrhs, s));
  BEM_TRY(bem_epilogue(o->h, o->nrhs, BEM_C128, in, out, 1, s));
  return BEM_OK;
}
}  // namespace

// the nrhs right-hand sides of one operator: column r is [r N, (r + 1) N)
int bem_gmres(bem_handle* h, int nrhs, int dtype, const void* b_in, void* x_out, double tol, int max_iter,
              int restart, int flags, int* iters_out, double* relres_out, cudaStream_t s) {
  std::vector<int64_t> off(nrhs), len(nrhs, h->nt);
  for (int r = 0; r < nrhs; ++r) off[r] = (int64_t)r * h->nt;
  OneOp ctx{h, nrhs};
  return bem_gmres_core(one_op_apply, &ctx, nrhs, (int64_t)nrhs * h->nt, off.data(), len.data(), dtype, b_in, x_out,
                        tol, max_iter, restart, flags, iters_out, relres_out, s);
}
