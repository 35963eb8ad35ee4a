// bem_chain.cu -- the adjoint chain of Section 2.2 and the topological
// derivative of Section 2.5 as single calls through the C ABI.  Each step is
// one of the library's own entry points (GMRES, off-surface evaluation, point
// sources, the T formula); the glue between them (p_obs = p_inc + D p, its
// conjugate as the adjoint weights, p = p_inc + D p and pa = phi + D pa at the
// field points) runs in the small kernels below.
#include "bem_common.cuh"

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// out[i] = base[i] - u[i] over n complex values (u in the handle's dtype),
// and optionally conj(out) into cj: the rigid body's representation formula
// p = p_inc + D p_surf, with u = -D p_surf as the evaluation returns it.
// out may be base (each thread reads its entry before writing it).
template <typename Ru>
__global__ void k_chain_combine(int64_t n, const Ru* __restrict__ u, const double* base, double* out,
                                double* __restrict__ cj) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double re = base[2 * i] - (double)u[2 * i], im = base[2 * i + 1] - (double)u[2 * i + 1];
  out[2 * i] = re;
  out[2 * i + 1] = im;
  if (cj) {
    cj[2 * i] = re;
    cj[2 * i + 1] = -im;
  }
}

static int combine(int dtype, int64_t n, const void* u, const double* base, double* out, double* cj, cudaStream_t s) {
  if (dtype == BEM_C128)
    k_chain_combine<double><<<nblk(n, 256), 256, 0, s>>>(n, (const double*)u, base, out, cj);
  else
    k_chain_combine<float><<<nblk(n, 256), 256, 0, s>>>(n, (const float*)u, base, out, cj);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

extern "C" {

int bem_state_adjoint(bem_handle* h, int dtype, const void* b, int nobs, const double* observers,
                      const double* incident_obs, double tol, int max_iter, int restart, int flags, void* p,
                      double* p_obs, double* weights, void* p_adj, int* iters, double* relres, void* stream) {
  bem_set_error("");
  if (!h) return bem_fail(BEM_ERR_INVALID_ARG, "handle is NULL");
  if (dtype != BEM_C64 && dtype != BEM_C128) return bem_fail(BEM_ERR_INVALID_ARG, "dtype must be BEM_C64 or BEM_C128");
  if (!b || !p || !p_adj || !observers || !incident_obs || !p_obs || !weights || !iters || !relres || nobs < 1)
    return bem_fail(BEM_ERR_INVALID_ARG, "buffers required, nobs >= 1");
  if (flags & BEM_GMRES_USE_X0) return bem_fail(BEM_ERR_INVALID_ARG, "the chain starts both solves from zero");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t esz = dtype == BEM_C128 ? 16 : 8;
  iters[0] = iters[1] = 0;
  relres[0] = relres[1] = 0.0;
  // state solve (1/2 I - D) p = b
  BEM_CUDA(cudaMemsetAsync(p, 0, esz * h->nt, s));
  BEM_TRY(bem_gmres_solve(h, 1, dtype, b, p, tol, max_iter, restart, flags, &iters[0], &relres[0], stream));
  // p(x_m) = p_inc(x_m) + (D p)(x_m); weights conj(p(x_m)) (f = 1/2 |p|^2)
  void* u = nullptr;
  void* badj = nullptr;
  int rc = BEM_OK;
  do {
    cudaError_t e = cudaMallocAsync(&u, esz * nobs, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&badj, esz * h->nt, s);
    if (e != cudaSuccess) {
      rc = bem_fail(e == cudaErrorMemoryAllocation ? BEM_ERR_OOM : BEM_ERR_CUDA, cudaGetErrorString(e));
      break;
    }
    rc = bem_eval_points(h, 1, dtype, p, nullptr, observers, nobs, u, 0, stream);
    if (rc != BEM_OK) break;
    rc = combine(dtype, nobs, u, incident_obs, p_obs, weights, s);
    if (rc != BEM_OK) break;
    // adjoint right-hand side sum_m conj(p(x_m)) G(c_i - x_m), adjoint solve
    rc = bem_point_sources(h, 1, dtype, nobs, observers, weights, badj, stream);
    if (rc != BEM_OK) break;
    e = cudaMemsetAsync(p_adj, 0, esz * h->nt, s);
    if (e != cudaSuccess) {
      rc = bem_fail(BEM_ERR_CUDA, cudaGetErrorString(e));
      break;
    }
    rc = bem_gmres_solve(h, 1, dtype, badj, p_adj, tol, max_iter, restart, flags, &iters[1], &relres[1], stream);
  } while (false);
  if (u) cudaFreeAsync(u, s);
  if (badj) cudaFreeAsync(badj, s);
  return rc;
}

int bem_topological_field(bem_handle* h, int dtype, const void* p, const void* p_adj, int nobs,
                          const double* observers, const double* weights, int64_t npoints, const double* points,
                          const double* incident, double c1, double c2, double* T, void* stream) {
  bem_set_error("");
  if (!h) return bem_fail(BEM_ERR_INVALID_ARG, "handle is NULL");
  if (dtype != BEM_C64 && dtype != BEM_C128) return bem_fail(BEM_ERR_INVALID_ARG, "dtype must be BEM_C64 or BEM_C128");
  if (!p || !p_adj || !observers || !weights || !points || !incident || !T || nobs < 1 || npoints < 1)
    return bem_fail(BEM_ERR_INVALID_ARG, "buffers required, nobs >= 1, npoints >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t esz = dtype == BEM_C128 ? 16 : 8;
  const int64_t nv = 4 * npoints;  // (value, d/dx, d/dy, d/dz) per point
  void* u = nullptr;
  double *state = nullptr, *adj = nullptr;
  int rc = BEM_OK;
  do {
    cudaError_t e = cudaMallocAsync(&u, esz * nv, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&state, 16 * nv, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&adj, 16 * nv, s);
    if (e != cudaSuccess) {
      rc = bem_fail(e == cudaErrorMemoryAllocation ? BEM_ERR_OOM : BEM_ERR_CUDA, cudaGetErrorString(e));
      break;
    }
    // state: p = p_inc + D p_surf with its gradient
    rc = bem_eval_points(h, 1, dtype, p, nullptr, points, npoints, u, BEM_EVAL_VALUE_GRADIENT, stream);
    if (rc != BEM_OK) break;
    rc = combine(dtype, nv, u, incident, state, nullptr, s);
    if (rc != BEM_OK) break;
    // adjoint: pa = phi + D pa_surf, phi the point sources at the observers
    rc = bem_point_source_field(1, nobs, observers, weights, npoints, points, h->k, BEM_EVAL_GRADIENT, adj, stream);
    if (rc != BEM_OK) break;
    rc = bem_eval_points(h, 1, dtype, p_adj, nullptr, points, npoints, u, BEM_EVAL_VALUE_GRADIENT, stream);
    if (rc != BEM_OK) break;
    rc = combine(dtype, nv, u, adj, adj, nullptr, s);
    if (rc != BEM_OK) break;
    rc = bem_topological_derivative(npoints, c1, c2, state, adj, T, stream);
  } while (false);
  for (void* q : {u, (void*)state, (void*)adj})
    if (q) cudaFreeAsync(q, s);
  return rc;
}

}  // extern "C"
