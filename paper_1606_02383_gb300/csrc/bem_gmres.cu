// bem_gmres.cu -- restarted GMRES for (1/2 I - D) x = b (Section 2.3, Eq. (GMRES)
// without the FEM coupling term; Section 3: GMRES with a relative tolerance).
//
// The core solves `ncol` independent systems in lockstep: column c is the
// complex segment [off[c], off[c] + len[c]) of one block vector of length M,
// and every iteration makes one apply of the whole block (a multi-rhs apply of
// one operator, or one batch apply of many operators).  Krylov vectors, dot
// products and updates are FP64 on the device; orthogonalisation is classical
// Gram-Schmidt applied twice (CGS2).
//
// Two drivers share the arithmetic.  By default a restart cycle is one CUDA
// graph: the Arnoldi steps run in a conditional WHILE node, the small
// Hessenberg least-squares problems (Givens rotations) are solved on the device
// and the host reads the residuals once per cycle.  The host-driven loop
// (BEM_GMRES_HOST_LOOP, and the fallback when no graph can be built) solves the
// small problems on the host and reads j+2 coefficients per column after every
// iteration.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "bem_common.cuh"

typedef std::complex<double> hz;
static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

#define GM_TILE 2048      // elements per dot-product work item, at least
#define GM_MAX_ITEMS 256  // dot-product work items per column, at most
#define GM_VSPLIT 8       // Krylov vectors are spread over this many blocks per work item

// Control block of the graph-resident cycles (below), read by the kernels of
// the captured Arnoldi step so that one captured body serves every step j.
struct GmCtl {
  int j;     // Arnoldi step within the cycle: V_0 .. V_j exist
  int jlim;  // steps allowed in this cycle: min(restart, max_iter - it)
  int it;    // iterations over all cycles
  int any;   // some column still active
};

// a count given by the host (fixed > 0) or the control block's j + add
__device__ __forceinline__ int gm_count(int fixed, const GmCtl* ctl, int add) {
  return fixed > 0 ? fixed : ctl->j + add;
}

// colof[off[c] + e] = c for every element of every column
__global__ void k_gm_colof(const int64_t* __restrict__ off, const int64_t* __restrict__ len, int* colof) {
  const int c = blockIdx.y;
  const int64_t n = len[c], o = off[c];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    colof[o + e] = c;
}

// Dot products conj(V_i) . w per column, i < nv.  Work item t is chunk
// item_k[t] of the nch[c] equal chunks of column c = item_col[t] (chunks of at
// least GM_TILE elements, so that short columns are not split into blocks that
// do little but reduce); partial[i * nitems + t] gets its sum.
__global__ void __launch_bounds__(256) k_gm_dots(int fixed_nv, const GmCtl* __restrict__ ctl, int nitems,
                                                 const int* __restrict__ item_col, const int* __restrict__ item_k,
                                                 const int* __restrict__ nch, const int64_t* __restrict__ off,
                                                 const int64_t* __restrict__ len, const double* __restrict__ V,
                                                 int64_t vstride, const double* __restrict__ w, double* partial) {
  const int nv = gm_count(fixed_nv, ctl, 1);
  const int t = blockIdx.x, c = item_col[t], k = item_k[t];
  const int64_t n = len[c], per = (n + nch[c] - 1) / nch[c];
  const int64_t a = k * per, b = min(n, a + per);
  const double2* ww = (const double2*)(w + 2 * off[c]);
  __shared__ double sh[2][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = blockIdx.y; i < nv; i += GM_VSPLIT) {
    const double2* v = (const double2*)(V + i * vstride + 2 * off[c]);
    double sre = 0.0, sim = 0.0;
#pragma unroll 4
    for (int64_t e = a + threadIdx.x; e < b; e += 256) {
      const double2 vv = v[e], x = ww[e];
      sre += vv.x * x.x + vv.y * x.y;
      sim += vv.x * x.y - vv.y * x.x;
    }
    for (int o = 16; o > 0; o >>= 1) {
      sre += __shfl_xor_sync(0xffffffffu, sre, o);
      sim += __shfl_xor_sync(0xffffffffu, sim, o);
    }
    if (lane == 0) {
      sh[0][warp] = sre;
      sh[1][warp] = sim;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double tr = 0.0, ti = 0.0;
      for (int q = 0; q < 8; ++q) {
        tr += sh[0][q];
        ti += sh[1][q];
      }
      partial[2 * ((int64_t)i * nitems + t)] = tr;
      partial[2 * ((int64_t)i * nitems + t) + 1] = ti;
    }
    __syncthreads();
  }
}

// out[c*mp1 + i] = sum over column c's work items, i < nv; one warp per (c, i)
__global__ void k_gm_reduce(int fixed_nv, const GmCtl* __restrict__ ctl, int ncol, int mp1, int nitems,
                            const int* __restrict__ item0, const int* __restrict__ nch,
                            const double* __restrict__ partial, double* out) {
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= (int64_t)ncol * mp1) return;
  const int c = (int)(wid / mp1), i = (int)(wid % mp1);
  if (i >= gm_count(fixed_nv, ctl, 1)) return;
  const double* p = partial + 2 * ((int64_t)i * nitems + item0[c]);
  double sre = 0.0, sim = 0.0;
  for (int t = lane; t < nch[c]; t += 32) {
    sre += p[2 * t];
    sim += p[2 * t + 1];
  }
  for (int o = 16; o > 0; o >>= 1) {
    sre += __shfl_xor_sync(0xffffffffu, sre, o);
    sim += __shfl_xor_sync(0xffffffffu, sim, o);
  }
  if (lane == 0) {
    out[2 * wid] = sre;
    out[2 * wid + 1] = sim;
  }
}

// w -= sum_{i < nv} coef[c*mp1 + i] V_i   on every element e of column c = colof[e]
__global__ void k_gm_orth(int64_t M, int fixed_nv, const GmCtl* __restrict__ ctl, int mp1,
                          const int* __restrict__ colof, const double* __restrict__ V, int64_t vstride,
                          const double* __restrict__ coef, double* w) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= M) return;
  const int c = colof[e], nv = gm_count(fixed_nv, ctl, 1);
  const double2* cf = (const double2*)coef + (int64_t)c * mp1;
  double2 x = ((const double2*)w)[e];
#pragma unroll 4
  for (int i = 0; i < nv; ++i) {
    const double2 q = cf[i], v = ((const double2*)(V + i * vstride))[e];
    x.x -= q.x * v.x - q.y * v.y;
    x.y -= q.x * v.y + q.y * v.x;
  }
  ((double2*)w)[e] = x;
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

// x += sum_{i < nv} y[c*mp1 + i] V_i
__global__ void k_gm_update_x(int64_t M, int fixed_nv, const GmCtl* __restrict__ ctl, int mp1,
                              const int* __restrict__ colof, const double* __restrict__ V, int64_t vstride,
                              const double* __restrict__ y, double* x) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= M) return;
  const int c = colof[e], nv = gm_count(fixed_nv, ctl, 0);
  const double2* yc = (const double2*)y + (int64_t)c * mp1;
  double2 acc = ((const double2*)x)[e];
#pragma unroll 4
  for (int i = 0; i < nv; ++i) {
    const double2 q = yc[i], v = ((const double2*)(V + i * vstride))[e];
    acc.x += q.x * v.x - q.y * v.y;
    acc.y += q.x * v.y + q.y * v.x;
  }
  ((double2*)x)[e] = acc;
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

// ------------------------------------------------ device-resident cycles --
// One restart cycle as one CUDA graph: the residual, its norm and the start
// of the cycle; a conditional WHILE node whose body is one Arnoldi step
// (apply, CGS2, norm, Givens rotations of every column); then the triangular
// solves and the update of x.  Every kernel of the body reads the step j from
// a control block in device memory, so one captured body serves every j, and
// the Givens kernel decides on the device whether the loop goes on.  The host
// reads the residuals once per cycle.
// dst = V_j (the apply's input)
__global__ void k_gmd_copy_vj(int64_t n, const GmCtl* __restrict__ ctl, const double* __restrict__ V, int64_t vstride,
                              double* dst) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < n) dst[e] = V[(int64_t)ctl->j * vstride + e];
}

// V_j = w * scale[column]
__global__ void k_gmd_scale(int64_t M, const GmCtl* __restrict__ ctl, const int* __restrict__ colof,
                            const double* __restrict__ w, const double* __restrict__ scale, double* V,
                            int64_t vstride) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= M) return;
  double s = scale[colof[e]];
  double* d = V + (int64_t)ctl->j * vstride;
  d[2 * e] = w[2 * e] * s;
  d[2 * e + 1] = w[2 * e + 1] * s;
}

__device__ __forceinline__ double gmd_bnorm(const double* nrm_b, int c) {
  double bn = sqrt(fmax(0.0, nrm_b[2 * c]));
  return bn > 0.0 ? bn : 1.0;
}

// Start of a cycle (one block): beta = |r0| per column, the active columns,
// 1 / beta for V_0, g = beta e_1; j = 0 and the step limit; the loop runs if
// some column is active.
__global__ void k_gmd_start(int ncol, int m, int max_iter, double tol, const double* __restrict__ nrm_r,
                            const double* __restrict__ nrm_b, GmCtl* ctl, int* active, int* ncols, double* relres,
                            double* scale, double* gg, int mp1, cudaGraphConditionalHandle cond) {
  __shared__ int any_s;
  if (threadIdx.x == 0) any_s = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
    const double beta = sqrt(fmax(0.0, nrm_r[2 * c]));
    relres[c] = beta / gmd_bnorm(nrm_b, c);
    const int act = relres[c] > tol && beta > 0.0;
    active[c] = act;
    ncols[c] = 0;
    scale[c] = act ? 1.0 / beta : 0.0;
    gg[2 * (int64_t)c * mp1] = beta;
    gg[2 * (int64_t)c * mp1 + 1] = 0.0;
    if (act) any_s = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int jlim = min(m, max_iter - ctl->it);
    ctl->j = 0;
    ctl->jlim = jlim;
    ctl->any = any_s;
    cudaGraphSetConditional(cond, (any_s && jlim > 0) ? 1u : 0u);
  }
}

// One Arnoldi step's small problem for every active column (one block, a
// thread per column): Hessenberg column j = coef + coef2 and |w|, the earlier
// rotations, a new rotation zeroing H[j+1][j], g updated; the column stops on
// |g[j+1]| / |b| <= tol or on breakdown.  Then j advances and the loop goes on
// while a column is active and j < jlim.
__global__ void k_gmd_givens(int ncol, int m, int mp1, double tol, const double* __restrict__ coef,
                             const double* __restrict__ coef2, const double* __restrict__ nrm_w,
                             const double* __restrict__ nrm_b, GmCtl* ctl, double* H, double* cs, double* sn,
                             double* gg, int* active, int* ncols, double* relres, double* scale,
                             cudaGraphConditionalHandle cond) {
  __shared__ int any_s;
  const int j = ctl->j;
  if (threadIdx.x == 0) any_s = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
    if (!active[c]) {
      scale[c] = 0.0;
      continue;
    }
    double* Hc = H + 2 * (int64_t)c * mp1 * m;
    double* csc = cs + (int64_t)c * m;
    double* snc = sn + 2 * (int64_t)c * m;
    double* g = gg + 2 * (int64_t)c * mp1;
#define HR(i, q) Hc[2 * ((int64_t)(i) * m + (q))]
#define HI(i, q) Hc[2 * ((int64_t)(i) * m + (q)) + 1]
    for (int i = 0; i <= j; ++i) {
      HR(i, j) = coef[2 * (c * mp1 + i)] + coef2[2 * (c * mp1 + i)];
      HI(i, j) = coef[2 * (c * mp1 + i) + 1] + coef2[2 * (c * mp1 + i) + 1];
    }
    const double hn = sqrt(fmax(0.0, nrm_w[2 * c]));
    HR(j + 1, j) = hn;
    HI(j + 1, j) = 0.0;
    for (int i = 0; i < j; ++i) {  // earlier rotations
      const double ar = HR(i, j), ai = HI(i, j), br = HR(i + 1, j), bi = HI(i + 1, j);
      const double c_ = csc[i], sr = snc[2 * i], si = snc[2 * i + 1];
      HR(i, j) = c_ * ar + (sr * br - si * bi);
      HI(i, j) = c_ * ai + (sr * bi + si * br);
      HR(i + 1, j) = -(sr * ar + si * ai) + c_ * br;  // -conj(s) a + c b
      HI(i + 1, j) = -(sr * ai - si * ar) + c_ * bi;
    }
    const double ar = HR(j, j), ai = HI(j, j);
    const double bq = hypot(HR(j + 1, j), HI(j + 1, j));
    const double aa = hypot(ar, ai);
    const double rho = hypot(aa, bq);
    double cj, sjr, sji;
    if (aa == 0.0) {
      cj = 0.0;
      sjr = 1.0;
      sji = 0.0;
    } else {
      cj = aa / rho;
      sjr = (ar / aa) * bq / rho;
      sji = (ai / aa) * bq / rho;
    }
    csc[j] = cj;
    snc[2 * j] = sjr;
    snc[2 * j + 1] = sji;
    HR(j, j) = cj * ar + sjr * bq;
    HI(j, j) = cj * ai + sji * bq;
    HR(j + 1, j) = 0.0;
    HI(j + 1, j) = 0.0;
    const double gr = g[2 * j], gi = g[2 * j + 1];
    g[2 * (j + 1)] = -(sjr * gr + sji * gi);  // -conj(s) g_j
    g[2 * (j + 1) + 1] = -(sjr * gi - sji * gr);
    g[2 * j] = cj * gr;
    g[2 * j + 1] = cj * gi;
    ncols[c] = j + 1;
    relres[c] = hypot(g[2 * (j + 1)], g[2 * (j + 1) + 1]) / gmd_bnorm(nrm_b, c);
    const bool breakdown = !(hn > 1e-14 * hypot(HR(j, j), HI(j, j)));
#undef HR
#undef HI
    if (relres[c] <= tol || breakdown) {
      active[c] = 0;
      scale[c] = 0.0;
    } else {
      scale[c] = 1.0 / hn;
      any_s = 1;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int jn = j + 1;
    ctl->j = jn;
    ctl->it += 1;
    ctl->any = any_s;
    cudaGraphSetConditional(cond, (any_s && jn < ctl->jlim) ? 1u : 0u);
  }
}

// y = R^-1 g per column (back substitution over its ncols columns); zeros up
// to the cycle's step count
__global__ void k_gmd_backsub(int ncol, int m, int mp1, const GmCtl* __restrict__ ctl, const double* __restrict__ H,
                              const double* __restrict__ gg, const int* __restrict__ ncols, double* y) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncol) return;
  const int k = ncols[c], jmax = ctl->j;
  const double* Hc = H + 2 * (int64_t)c * mp1 * m;
  const double* g = gg + 2 * (int64_t)c * mp1;
  double* yc = y + 2 * (int64_t)c * mp1;
  for (int i = k - 1; i >= 0; --i) {
    double accr = g[2 * i], acci = g[2 * i + 1];
    for (int q = i + 1; q < k; ++q) {
      const double hr = Hc[2 * ((int64_t)i * m + q)], hi = Hc[2 * ((int64_t)i * m + q) + 1];
      accr -= hr * yc[2 * q] - hi * yc[2 * q + 1];
      acci -= hr * yc[2 * q + 1] + hi * yc[2 * q];
    }
    const double dr = Hc[2 * ((int64_t)i * m + i)], di = Hc[2 * ((int64_t)i * m + i) + 1];
    const double den = dr * dr + di * di;
    yc[2 * i] = (accr * dr + acci * di) / den;
    yc[2 * i + 1] = (acci * dr - accr * di) / den;
  }
  for (int i = k; i < jmax; ++i) yc[2 * i] = yc[2 * i + 1] = 0.0;
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
  int mp1;                             // restart + 1: row stride of coef and y
  int nitems;                          // dot-product work items over all columns
  int *item_col, *item_k, *nch, *item0;  // per item: column, chunk; per column: chunks, first item
};

// norms of the ncol columns of `w` into a host array (synchronises)
int gm_norms(GmCore& g, const double* w, std::vector<double>& out) {
  k_gm_dots<<<g.nitems, 256, 0, g.s>>>(1, nullptr, g.nitems, g.item_col, g.item_k, g.nch, g.d_off, g.d_len, w, 0, w,
                                      g.partial);
  k_gm_reduce<<<nblk(32 * (int64_t)g.ncol, 128), 128, 0, g.s>>>(1, nullptr, g.ncol, 1, g.nitems, g.item0, g.nch,
                                                                 g.partial, g.nrm);
  std::vector<double> t(2 * (size_t)g.ncol);
  BEM_CUDA(cudaMemcpyAsync(t.data(), g.nrm, t.size() * sizeof(double), cudaMemcpyDeviceToHost, g.s));
  BEM_CUDA(cudaStreamSynchronize(g.s));
  out.resize(g.ncol);
  for (int c = 0; c < g.ncol; ++c) out[c] = std::sqrt(std::max(0.0, t[2 * c]));
  return BEM_OK;
}

}  // namespace

// device arrays of the graph-resident cycles
struct GmDev {
  GmCtl* ctl;
  double *H, *cs, *sn, *gg, *relres, *nrmb, *vin;
  int *active, *ncols;
};

// Captures one restart cycle into an executable graph (see the kernels above).
// `capply` must issue its work on the stream it is given without
// synchronising or allocating; it may fork onto other streams and join them
// back.  The cycle's outer part (residual, start, WHILE node, update of x) is
// captured first and its capture ended before the loop body is captured into
// the WHILE node's child graph, so that streams joined by one capture are free
// again for the other.  Every capture is closed on every return path.
static int gm_graph_build(GmCore& g, GmDev& d, bem_gm_apply_fn capply, int m, int max_iter, double tol,
                          cudaStream_t cs, cudaStream_t cs2, cudaGraphExec_t* exec) {
  const int ncol = g.ncol, mp1 = m + 1;
  const int64_t M = g.M, tot = 2 * M;
  const unsigned gvec = nblk(M, 256);
  cudaGraph_t body = nullptr;
  cudaGraphConditionalHandle cond;
  // outer part
  BEM_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  auto outer = [&]() -> int {
    cudaStreamCaptureStatus st;
    cudaGraph_t cg = nullptr;
    BEM_CUDA(cudaStreamGetCaptureInfo(cs, &st, nullptr, &cg, nullptr, nullptr, nullptr));
    BEM_CUDA(cudaGraphConditionalHandleCreate(&cond, cg, 0, cudaGraphCondAssignDefault));
    // r0 = b - A x, |r0|, start of the cycle, V_0
    BEM_TRY(capply(g.ctx, g.xx, g.w, cs));
    k_gm_sub<<<nblk(tot, 256), 256, 0, cs>>>(tot, g.bb, g.w, g.w);
    k_gm_dots<<<g.nitems, 256, 0, cs>>>(1, nullptr, g.nitems, g.item_col, g.item_k, g.nch, g.d_off, g.d_len, g.w, 0,
                                        g.w, g.partial);
    k_gm_reduce<<<nblk(32 * (int64_t)ncol, 128), 128, 0, cs>>>(1, nullptr, ncol, 1, g.nitems, g.item0, g.nch,
                                                               g.partial, g.nrm);
    k_gmd_start<<<1, 256, 0, cs>>>(ncol, m, max_iter, tol, g.nrm, d.nrmb, d.ctl, d.active, d.ncols, d.relres,
                                   g.scale, d.gg, mp1, cond);
    k_gmd_scale<<<gvec, 256, 0, cs>>>(M, d.ctl, g.colof, g.w, g.scale, g.V, g.vstride);
    BEM_CUDA(cudaGetLastError());
    // the Arnoldi loop: a WHILE node after everything captured so far
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    BEM_CUDA(cudaStreamGetCaptureInfo(cs, &st, nullptr, &cg, &deps, nullptr, &ndeps));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    BEM_CUDA(cudaGraphAddNode(&wnode, cg, deps, nullptr, ndeps, &cp));
    body = cp.conditional.phGraph_out[0];
    BEM_CUDA(cudaStreamUpdateCaptureDependencies(cs, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    // x += V y
    k_gmd_backsub<<<nblk(ncol, 64), 64, 0, cs>>>(ncol, m, mp1, d.ctl, d.H, d.gg, d.ncols, g.y);
    k_gm_update_x<<<gvec, 256, 0, cs>>>(M, 0, d.ctl, mp1, g.colof, g.V, g.vstride, g.y, g.xx);
    BEM_CUDA(cudaGetLastError());
    return BEM_OK;
  };
  int rc = outer();
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &graph);
  if (rc == BEM_OK && e != cudaSuccess)
    rc = bem_fail(BEM_ERR_CUDA, std::string("GMRES graph capture: ") + cudaGetErrorString(e));
  // the loop body, captured into the WHILE node's graph
  if (rc == BEM_OK) {
    e = cudaStreamBeginCaptureToGraph(cs2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) rc = bem_fail(BEM_ERR_CUDA, std::string("GMRES body capture: ") + cudaGetErrorString(e));
  }
  if (rc == BEM_OK) {
    auto inner = [&]() -> int {
      k_gmd_copy_vj<<<nblk(tot, 256), 256, 0, cs2>>>(tot, d.ctl, g.V, g.vstride, d.vin);
      BEM_TRY(capply(g.ctx, d.vin, g.w, cs2));
      const dim3 gd(g.nitems, GM_VSPLIT);
      const unsigned gr = nblk(32 * (int64_t)ncol * mp1, 128);
      k_gm_dots<<<gd, 256, 0, cs2>>>(0, d.ctl, g.nitems, g.item_col, g.item_k, g.nch, g.d_off, g.d_len, g.V,
                                     g.vstride, g.w, g.partial);
      k_gm_reduce<<<gr, 128, 0, cs2>>>(0, d.ctl, ncol, mp1, g.nitems, g.item0, g.nch, g.partial, g.coef);
      k_gm_orth<<<gvec, 256, 0, cs2>>>(M, 0, d.ctl, mp1, g.colof, g.V, g.vstride, g.coef, g.w);
      k_gm_dots<<<gd, 256, 0, cs2>>>(0, d.ctl, g.nitems, g.item_col, g.item_k, g.nch, g.d_off, g.d_len, g.V,
                                     g.vstride, g.w, g.partial);
      k_gm_reduce<<<gr, 128, 0, cs2>>>(0, d.ctl, ncol, mp1, g.nitems, g.item0, g.nch, g.partial, g.coef2);
      k_gm_orth<<<gvec, 256, 0, cs2>>>(M, 0, d.ctl, mp1, g.colof, g.V, g.vstride, g.coef2, g.w);
      k_gm_dots<<<g.nitems, 256, 0, cs2>>>(1, nullptr, g.nitems, g.item_col, g.item_k, g.nch, g.d_off, g.d_len, g.w, 0,
                                          g.w, g.partial);
      k_gm_reduce<<<nblk(32 * (int64_t)ncol, 128), 128, 0, cs2>>>(1, nullptr, ncol, 1, g.nitems, g.item0, g.nch,
                                                                 g.partial, g.nrm);
      k_gmd_givens<<<1, 256, 0, cs2>>>(ncol, m, mp1, tol, g.coef, g.coef2, g.nrm, d.nrmb, d.ctl, d.H, d.cs, d.sn,
                                       d.gg, d.active, d.ncols, d.relres, g.scale, cond);
      k_gmd_scale<<<gvec, 256, 0, cs2>>>(M, d.ctl, g.colof, g.w, g.scale, g.V, g.vstride);
      BEM_CUDA(cudaGetLastError());
      return BEM_OK;
    };
    rc = inner();
    cudaGraph_t bg = nullptr;
    e = cudaStreamEndCapture(cs2, &bg);
    if (rc == BEM_OK && e != cudaSuccess)
      rc = bem_fail(BEM_ERR_CUDA, std::string("GMRES body capture: ") + cudaGetErrorString(e));
  }
  if (rc == BEM_OK) {
    e = cudaGraphInstantiate(exec, graph, 0);
    if (e != cudaSuccess) rc = bem_fail(BEM_ERR_CUDA, std::string("GMRES graph instantiate: ") + cudaGetErrorString(e));
  }
  if (graph) cudaGraphDestroy(graph);
  if (rc != BEM_OK) cudaGetLastError();  // leave no launch error behind for the host-loop fallback
  return rc;
}

struct GmStreams {
  cudaStream_t cs = nullptr, cs2 = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~GmStreams() {
    if (exec) cudaGraphExecDestroy(exec);
    if (cs) cudaStreamDestroy(cs);
    if (cs2) cudaStreamDestroy(cs2);
  }
};

int bem_gmres_core(bem_gm_apply_fn apply, bem_gm_apply_fn capture_apply, void* ctx, int ncol, int64_t M,
                   const int64_t* off, const int64_t* len, int dtype, const void* b_in, void* x_out, double tol, int max_iter, int restart, int flags,
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
  // dot-product work items: chunks of at least GM_TILE elements, at most GM_MAX_ITEMS per column
  std::vector<int> nch(ncol), item0(ncol), item_col, item_k;
  for (int c = 0; c < ncol; ++c) {
    nch[c] = (int)std::min<int64_t>(GM_MAX_ITEMS, std::max<int64_t>(1, (len[c] + GM_TILE - 1) / GM_TILE));
    item0[c] = (int)item_col.size();
    for (int k = 0; k < nch[c]; ++k) {
      item_col.push_back(c);
      item_k.push_back(k);
    }
  }
  g.mp1 = m + 1;
  g.nitems = (int)item_col.size();
  BEM_TRY(sc_.get(&g.item_col, (size_t)g.nitems));
  BEM_TRY(sc_.get(&g.item_k, (size_t)g.nitems));
  BEM_TRY(sc_.get(&g.nch, (size_t)ncol));
  BEM_TRY(sc_.get(&g.item0, (size_t)ncol));
  BEM_TRY(sc_.get(&g.partial, (size_t)g.nitems * (m + 1) * 2));
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
  BEM_CUDA(cudaMemcpyAsync(g.item_col, item_col.data(), g.nitems * sizeof(int), cudaMemcpyHostToDevice, s));
  BEM_CUDA(cudaMemcpyAsync(g.item_k, item_k.data(), g.nitems * sizeof(int), cudaMemcpyHostToDevice, s));
  BEM_CUDA(cudaMemcpyAsync(g.nch, nch.data(), ncol * sizeof(int), cudaMemcpyHostToDevice, s));
  BEM_CUDA(cudaMemcpyAsync(g.item0, item0.data(), ncol * sizeof(int), cudaMemcpyHostToDevice, s));
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
  bool graph_done = false;
  if (capture_apply && !(flags & BEM_GMRES_HOST_LOOP)) {
    // device-resident cycles: one graph launch and one small read per cycle
    GmDev d;
    const int mp1 = m + 1;
    BEM_TRY(sc_.get(&d.ctl, 1));
    BEM_TRY(sc_.get(&d.H, (size_t)ncol * mp1 * m * 2));
    BEM_TRY(sc_.get(&d.cs, (size_t)ncol * m));
    BEM_TRY(sc_.get(&d.sn, (size_t)ncol * m * 2));
    BEM_TRY(sc_.get(&d.gg, (size_t)ncol * mp1 * 2));
    BEM_TRY(sc_.get(&d.relres, (size_t)ncol));
    BEM_TRY(sc_.get(&d.nrmb, (size_t)ncol * 2));
    BEM_TRY(sc_.get(&d.vin, 2 * (size_t)M));
    BEM_TRY(sc_.get(&d.active, (size_t)ncol));
    BEM_TRY(sc_.get(&d.ncols, (size_t)ncol));
    BEM_CUDA(cudaMemcpyAsync(d.nrmb, g.nrm, 2 * ncol * sizeof(double), cudaMemcpyDeviceToDevice, s));  // |b|^2
    BEM_CUDA(cudaMemsetAsync(d.ctl, 0, sizeof(GmCtl), s));
    BEM_CUDA(cudaStreamSynchronize(s));  // the scratch is ready before the captured work can run
    GmStreams gs;
    BEM_CUDA(cudaStreamCreateWithFlags(&gs.cs, cudaStreamNonBlocking));
    BEM_CUDA(cudaStreamCreateWithFlags(&gs.cs2, cudaStreamNonBlocking));
    int rc = gm_graph_build(g, d, capture_apply, m, max_iter, tol, gs.cs, gs.cs2, &gs.exec);
    if (rc != BEM_OK && (flags & BEM_GMRES_GRAPH_ONLY)) return rc;
    if (rc == BEM_OK) {
      std::vector<double> rr(ncol);
      while (it_total < max_iter && !all_conv) {
        BEM_CUDA(cudaGraphLaunch(gs.exec, s));
        GmCtl hc;
        BEM_CUDA(cudaMemcpyAsync(&hc, d.ctl, sizeof(GmCtl), cudaMemcpyDeviceToHost, s));
        BEM_CUDA(cudaMemcpyAsync(rr.data(), d.relres, ncol * sizeof(double), cudaMemcpyDeviceToHost, s));
        BEM_CUDA(cudaStreamSynchronize(s));
        it_total = hc.it;
        all_conv = true;
        for (int c = 0; c < ncol; ++c) {
          relres[c] = rr[c];
          if (!(rr[c] <= tol)) all_conv = false;
        }
        if (hc.j == 0) break;  // no column could take a step (non-finite residual)
      }
      graph_done = true;
    }
  }
  while (!graph_done && it_total < max_iter && !all_conv) {
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
      const dim3 gd(g.nitems, GM_VSPLIT);
      const unsigned gr = nblk(32 * (int64_t)ncol * g.mp1, 128);
      k_gm_dots<<<gd, 256, 0, s>>>(nv, nullptr, g.nitems, g.item_col, g.item_k, g.nch, g.d_off, g.d_len, g.V,
                                   g.vstride, g.w, g.partial);
      k_gm_reduce<<<gr, 128, 0, s>>>(nv, nullptr, ncol, g.mp1, g.nitems, g.item0, g.nch, g.partial, g.coef);
      k_gm_orth<<<gvec, 256, 0, s>>>(M, nv, nullptr, g.mp1, g.colof, g.V, g.vstride, g.coef, g.w);
      k_gm_dots<<<gd, 256, 0, s>>>(nv, nullptr, g.nitems, g.item_col, g.item_k, g.nch, g.d_off, g.d_len, g.V,
                                   g.vstride, g.w, g.partial);
      k_gm_reduce<<<gr, 128, 0, s>>>(nv, nullptr, ncol, g.mp1, g.nitems, g.item0, g.nch, g.partial, g.coef2);
      k_gm_orth<<<gvec, 256, 0, s>>>(M, nv, nullptr, g.mp1, g.colof, g.V, g.vstride, g.coef2, g.w);
      BEM_CUDA(cudaGetLastError());
      std::vector<double> hc(2 * (size_t)g.mp1 * ncol), hc2(2 * (size_t)g.mp1 * ncol);
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
          Hc[(size_t)i * m + j] = hz(hc[2 * (c * g.mp1 + i)] + hc2[2 * (c * g.mp1 + i)],
                                     hc[2 * (c * g.mp1 + i) + 1] + hc2[2 * (c * g.mp1 + i) + 1]);
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
      std::vector<double> yv(2 * (size_t)ncol * g.mp1, 0.0);
      for (int c = 0; c < ncol; ++c) {
        int k = ncols[c];
        std::vector<hz> yy(k);
        for (int i = k - 1; i >= 0; --i) {
          hz acc = gg[c][i];
          for (int q = i + 1; q < k; ++q) acc -= H[c][(size_t)i * m + q] * yy[q];
          yy[i] = acc / H[c][(size_t)i * m + i];
        }
        for (int i = 0; i < k; ++i) {
          yv[2 * (c * g.mp1 + i)] = yy[i].real();
          yv[2 * (c * g.mp1 + i) + 1] = yy[i].imag();
        }
      }
      BEM_CUDA(cudaMemcpyAsync(g.y, yv.data(), yv.size() * sizeof(double), cudaMemcpyHostToDevice, s));
      k_gm_update_x<<<gvec, 256, 0, s>>>(M, nvmax, nullptr, g.mp1, g.colof, g.V, g.vstride, g.y, g.xx);
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
// the same work for stream capture: the stage timers (events) stay off
int one_op_apply_capture(void* ctx, const double* in, double* out, cudaStream_t s) {
  OneOp* o = (OneOp*)ctx;
  const int prof = o->h->prof_on;
  o->h->prof_on = 0;
  const int rc = one_op_apply(ctx, in, out, s);
  o->h->prof_on = prof;
  return rc;
}
}  // namespace

// ------------------------------------------------------ coupled operator --
// Eq. (GMRES): (1/2 I - D + S C) x.  The caller's callback computes y = C x
// from the vector copied into its buffer cx (steps 2(a), 2(b)); one FMM apply
// with both densities gives (1/2 I - D) x + S y (step 2(c)).
namespace {
struct CoupledOp {
  bem_handle* h;
  int nrhs;
  bem_coupling_fn cb;
  void* cb_ctx;
  double* cx;
  double* cy;
};
int coupled_apply(void* ctx, const double* in, double* out, cudaStream_t s) {
  CoupledOp* o = (CoupledOp*)ctx;
  const size_t bytes = (size_t)o->nrhs * o->h->nt * 2 * sizeof(double);
  BEM_CUDA(cudaMemcpyAsync(o->cx, in, bytes, cudaMemcpyDeviceToDevice, s));
  const int rc = o->cb(o->cb_ctx, o->nrhs, (void*)s);
  if (rc != 0) return bem_fail(BEM_ERR_CALLBACK, "coupling callback returned " + std::to_string(rc));
  BEM_TRY(bem_prologue(o->h, o->nrhs, BEM_C128, in, o->cy, s));
  BEM_TRY(bem_apply_sorted(o->h, o->nrhs, s));
  BEM_TRY(bem_epilogue(o->h, o->nrhs, BEM_C128, in, out, 1, s));
  return BEM_OK;
}
}  // namespace

int bem_gmres_coupled(bem_handle* h, int nrhs, int dtype, const void* b_in, void* x_out, double tol, int max_iter,
                      int restart, bem_coupling_fn cb, void* cb_ctx, double* cx, double* cy, int flags,
                      int* iters_out, double* relres_out, cudaStream_t s) {
  std::vector<int64_t> off(nrhs), len(nrhs, h->nt);
  for (int r = 0; r < nrhs; ++r) off[r] = (int64_t)r * h->nt;
  CoupledOp ctx{h, nrhs, cb, cb_ctx, cx, cy};
  return bem_gmres_core(coupled_apply, nullptr, &ctx, nrhs, (int64_t)nrhs * h->nt, off.data(), len.data(), dtype,
                        b_in, x_out, tol, max_iter, restart, flags | BEM_GMRES_HOST_LOOP, iters_out, relres_out, s);
}

// the nrhs right-hand sides of one operator: column r is [r N, (r + 1) N)
int bem_gmres(bem_handle* h, int nrhs, int dtype, const void* b_in, void* x_out, double tol, int max_iter,
              int restart, int flags, int* iters_out, double* relres_out, cudaStream_t s) {
  std::vector<int64_t> off(nrhs), len(nrhs, h->nt);
  for (int r = 0; r < nrhs; ++r) off[r] = (int64_t)r * h->nt;
  OneOp ctx{h, nrhs};
  return bem_gmres_core(one_op_apply, one_op_apply_capture, &ctx, nrhs, (int64_t)nrhs * h->nt, off.data(), len.data(), dtype, b_in, x_out,
                        tol, max_iter, restart, flags, iters_out, relres_out, s);
}
