// bem_levelset.cu -- one step of the level-set update of Section 2.4 on the
// lattice that carries phi: the fictitious-time reaction-diffusion equation
//   d phi / dt = F + tau L^2 lap phi,  F = -C T_Omega where phi <= 0 (the fluid),
//                                      F =  C T_Omegac where phi > 0 (the body),
// with phi = phi_bar on the boundary of the design box.  Discretisation (the
// reading the oracle states): Q1 elements on the lattice's voxels, implicit
// in the diffusion and explicit in F,
//   (M / dt + tau L^2 K) phi_new = M (phi / dt + F)   on the interior nodes,
// then phi_new clamped to [-1, 1].
//
// On a uniform lattice the assembled Q1 mass and stiffness are tensor
// products of the 1-D hat-function matrices, m = h [1/6, 2/3, 1/6] and
// k = [-1, 2, -1] / h:  M = m x m x m,  K = k x m x m + m x k x m + m x m x k,
// so A = M / dt + tau L^2 K is a 27-point stencil with
//   A(d) = m(dx) m(dy) m(dz) / dt + tau L^2 [k(dx) m(dy) m(dz) + m(dx) k(dy) m(dz) + m(dx) m(dy) k(dz)].
// Every interior node has its full stencil (all 8 voxels around it lie in
// the lattice).  The interior system is symmetric positive definite and is
// solved matrix-free by conjugate gradients in FP64 with the iterate's
// scalars on the device; the host reads the residual every few iterations.
#include <cmath>

#include "bem_common.cuh"

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

struct LsGrid {
  int n0, n1, n2;
  double w[27];  // stencil weights, index (dx + 1) * 9 + (dy + 1) * 3 + (dz + 1)
};

__device__ __forceinline__ bool ls_boundary(const LsGrid& g, int i, int j, int k) {
  return i == 0 || j == 0 || k == 0 || i == g.n0 - 1 || j == g.n1 - 1 || k == g.n2 - 1;
}

// y = A x on the interior nodes (0 on the boundary); x is a full lattice vector
__global__ void k_ls_apply(LsGrid g, const double* __restrict__ x, double* __restrict__ y) {
  const int64_t n = (int64_t)g.n0 * g.n1 * g.n2;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int k = (int)(idx % g.n2), j = (int)((idx / g.n2) % g.n1), i = (int)(idx / ((int64_t)g.n1 * g.n2));
  if (ls_boundary(g, i, j, k)) {
    y[idx] = 0.0;
    return;
  }
  const int64_t s1 = g.n2, s0 = (int64_t)g.n1 * g.n2;
  double acc = 0.0;
#pragma unroll
  for (int a = -1; a <= 1; ++a)
#pragma unroll
    for (int b = -1; b <= 1; ++b)
#pragma unroll
      for (int c = -1; c <= 1; ++c) acc += g.w[(a + 1) * 9 + (b + 1) * 3 + (c + 1)] * x[idx + a * s0 + b * s1 + c];
  y[idx] = acc;
}

// v = phi / dt + F on every node (the vector the mass matrix multiplies), and
// the boundary vector xb (phi_bar on the boundary, 0 inside), the initial
// iterate x (phi inside, 0 on the boundary)
__global__ void k_ls_prepare(LsGrid g, const double* __restrict__ phi, const double* __restrict__ t_in,
                             const double* __restrict__ t_out, double dt, double C, double phi_bar,
                             double* __restrict__ v, double* __restrict__ xb, double* __restrict__ x) {
  const int64_t n = (int64_t)g.n0 * g.n1 * g.n2;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int k = (int)(idx % g.n2), j = (int)((idx / g.n2) % g.n1), i = (int)(idx / ((int64_t)g.n1 * g.n2));
  const double p = phi[idx];
  const double F = p <= 0.0 ? -C * t_in[idx] : C * t_out[idx];
  v[idx] = p / dt + F;
  const bool bnd = ls_boundary(g, i, j, k);
  xb[idx] = bnd ? phi_bar : 0.0;
  x[idx] = bnd ? 0.0 : p;
}

// y = M v restricted to the interior: the stencil of the mass matrix alone
__global__ void k_ls_mass(LsGrid gm, const double* __restrict__ v, double* __restrict__ y) {
  const int64_t n = (int64_t)gm.n0 * gm.n1 * gm.n2;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int k = (int)(idx % gm.n2), j = (int)((idx / gm.n2) % gm.n1), i = (int)(idx / ((int64_t)gm.n1 * gm.n2));
  if (ls_boundary(gm, i, j, k)) {
    y[idx] = 0.0;
    return;
  }
  const int64_t s1 = gm.n2, s0 = (int64_t)gm.n1 * gm.n2;
  double acc = 0.0;
#pragma unroll
  for (int a = -1; a <= 1; ++a)
#pragma unroll
    for (int b = -1; b <= 1; ++b)
#pragma unroll
      for (int c = -1; c <= 1; ++c) acc += gm.w[(a + 1) * 9 + (b + 1) * 3 + (c + 1)] * v[idx + a * s0 + b * s1 + c];
  y[idx] = acc;
}

// block sum of a * b into *out (out zeroed by the caller)
__global__ void k_ls_dot(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* out) {
  __shared__ double sm[256];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += a[i] * b[i];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, sm[0]);
}

// r = rhs - A x (both interior; rhs = M v - A xb computed before); p = r
__global__ void k_ls_residual(int64_t n, const double* __restrict__ Mv, const double* __restrict__ Axb,
                              const double* __restrict__ Ax, double* __restrict__ rhs, double* __restrict__ r,
                              double* __restrict__ p) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double b = Mv[i] - Axb[i];
  rhs[i] = b;
  r[i] = b - Ax[i];
  p[i] = r[i];
}

// scalars s: [0] r.r, [1] p.Ap, [2] r.r of the new residual, [3] ||rhs||^2
// x += alpha p, r -= alpha Ap, with alpha = s[0] / s[1] read on the device
__global__ void k_ls_update(int64_t n, const double* __restrict__ s, const double* __restrict__ p,
                            const double* __restrict__ Ap, double* __restrict__ x, double* __restrict__ r) {
  const double pap = s[1];
  const double alpha = pap != 0.0 ? s[0] / pap : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    r[i] -= alpha * Ap[i];
  }
}

// p = r + beta p with beta = s[2] / s[0]; then s[0] = s[2], s[1] = s[2] = 0
__global__ void k_ls_direction(int64_t n, double* __restrict__ s, const double* __restrict__ r, double* __restrict__ p) {
  const double beta = s[0] != 0.0 ? s[2] / s[0] : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = r[i] + beta * p[i];
}

__global__ void k_ls_roll(double* s) {
  s[0] = s[2];
  s[1] = 0.0;
  s[2] = 0.0;
}

// phi_new = clamp(x inside, phi_bar on the boundary)
__global__ void k_ls_finish(int64_t n, const double* __restrict__ x, const double* __restrict__ xb, LsGrid g,
                            double* __restrict__ out) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int k = (int)(idx % g.n2), j = (int)((idx / g.n2) % g.n1), i = (int)(idx / ((int64_t)g.n1 * g.n2));
  const double v = ls_boundary(g, i, j, k) ? xb[idx] : x[idx];
  out[idx] = fmin(1.0, fmax(-1.0, v));
}

static void ls_weights(double h, double a_m, double a_k, double* w) {
  // 1-D factors: m = h [1/6, 2/3, 1/6], k = [-1, 2, -1] / h
  const double m[3] = {h / 6.0, 2.0 * h / 3.0, h / 6.0};
  const double kk[3] = {-1.0 / h, 2.0 / h, -1.0 / h};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c)
        w[a * 9 + b * 3 + c] =
            a_m * m[a] * m[b] * m[c] + a_k * (kk[a] * m[b] * m[c] + m[a] * kk[b] * m[c] + m[a] * m[b] * kk[c]);
}

extern "C" int bem_levelset_step(int n0, int n1, int n2, const double* phi, const double* t_omega,
                                 const double* t_omegac, double h, double dt, double C, double tau, double L,
                                 double phi_bar, double tol, int max_iter, double* phi_out, int* iters_out,
                                 double* relres_out, void* stream) {
  bem_set_error("");
  if (n0 < 1 || n1 < 1 || n2 < 1) return bem_fail(BEM_ERR_INVALID_ARG, "lattice sizes must be >= 1");
  if ((int64_t)n0 * n1 * n2 > ((int64_t)1 << 31)) return bem_fail(BEM_ERR_INVALID_ARG, "lattice above 2^31 nodes");
  if (!phi || !t_omega || !t_omegac || !phi_out) return bem_fail(BEM_ERR_INVALID_ARG, "phi, T and phi_out required");
  if (!(h > 0.0) || !(dt > 0.0) || !(tau >= 0.0) || !std::isfinite(h * dt * tau * L * C * phi_bar))
    return bem_fail(BEM_ERR_INVALID_ARG, "need h > 0, dt > 0, tau >= 0 and finite parameters");
  if (!(tol > 0.0) || max_iter < 1) return bem_fail(BEM_ERR_INVALID_ARG, "need tol > 0 and max_iter >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = (int64_t)n0 * n1 * n2;
  LsGrid gA, gM;
  gA.n0 = gM.n0 = n0;
  gA.n1 = gM.n1 = n1;
  gA.n2 = gM.n2 = n2;
  ls_weights(h, 1.0 / dt, tau * L * L, gA.w);
  ls_weights(h, 1.0, 0.0, gM.w);
  double* buf = nullptr;
  const size_t nb = 9 * (size_t)n + 8;
  cudaError_t e = cudaMallocAsync((void**)&buf, nb * sizeof(double), s);
  if (e != cudaSuccess)
    return bem_fail(e == cudaErrorMemoryAllocation ? BEM_ERR_OOM : BEM_ERR_CUDA, cudaGetErrorString(e));
  double *v = buf, *xb = v + n, *x = xb + n, *Mv = x + n, *Axb = Mv + n, *rhs = Axb + n, *r = rhs + n, *p = r + n,
         *Ap = p + n, *sc = Ap + n;
  int rc = BEM_OK;
  int it = 0;
  double rel = 0.0;
  const unsigned g1 = nblk(n, 256);
  const unsigned gr = (unsigned)std::min<int64_t>(g1, 1024);
  auto chk = [&]() {
    const cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess && rc == BEM_OK) rc = bem_fail(BEM_ERR_CUDA, cudaGetErrorString(ce));
    return rc == BEM_OK;
  };
  do {
    k_ls_prepare<<<g1, 256, 0, s>>>(gA, phi, t_omega, t_omegac, dt, C, phi_bar, v, xb, x);
    k_ls_mass<<<g1, 256, 0, s>>>(gM, v, Mv);
    k_ls_apply<<<g1, 256, 0, s>>>(gA, xb, Axb);
    k_ls_apply<<<g1, 256, 0, s>>>(gA, x, Ap);
    k_ls_residual<<<g1, 256, 0, s>>>(n, Mv, Axb, Ap, rhs, r, p);
    if (cudaMemsetAsync(sc, 0, 8 * sizeof(double), s) != cudaSuccess) {
      rc = bem_fail(BEM_ERR_CUDA, "memset");
      break;
    }
    k_ls_dot<<<gr, 256, 0, s>>>(n, r, r, sc);
    k_ls_dot<<<gr, 256, 0, s>>>(n, rhs, rhs, sc + 3);
    if (!chk()) break;
    double hs[4];
    if (cudaMemcpyAsync(hs, sc, 4 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      rc = bem_fail(BEM_ERR_CUDA, "reading the residual");
      break;
    }
    const double bnorm = std::sqrt(hs[3]);
    if (!std::isfinite(hs[0]) || !std::isfinite(hs[3])) {
      rc = bem_fail(BEM_ERR_NUMERIC, "non-finite right-hand side");
      break;
    }
    rel = bnorm > 0.0 ? std::sqrt(hs[0]) / bnorm : 0.0;
    // conjugate gradients; the residual is read every 8 iterations
    while (rel > tol && it < max_iter) {
      const int chunk = std::min(8, max_iter - it);
      for (int c = 0; c < chunk; ++c) {
        k_ls_apply<<<g1, 256, 0, s>>>(gA, p, Ap);
        k_ls_dot<<<gr, 256, 0, s>>>(n, p, Ap, sc + 1);
        k_ls_update<<<gr, 256, 0, s>>>(n, sc, p, Ap, x, r);
        k_ls_dot<<<gr, 256, 0, s>>>(n, r, r, sc + 2);
        k_ls_direction<<<gr, 256, 0, s>>>(n, sc, r, p);
        k_ls_roll<<<1, 1, 0, s>>>(sc);
      }
      it += chunk;
      if (!chk()) break;
      if (cudaMemcpyAsync(hs, sc, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        rc = bem_fail(BEM_ERR_CUDA, "reading the residual");
        break;
      }
      if (!std::isfinite(hs[0])) {
        rc = bem_fail(BEM_ERR_NUMERIC, "non-finite residual");
        break;
      }
      rel = bnorm > 0.0 ? std::sqrt(hs[0]) / bnorm : 0.0;
    }
    if (rc != BEM_OK) break;
    k_ls_finish<<<g1, 256, 0, s>>>(n, x, xb, gA, phi_out);
    if (!chk()) break;
    if (rel > tol) rc = bem_fail(BEM_ERR_NOT_CONVERGED, "level-set step: conjugate gradients reached max_iter");
  } while (false);
  cudaFreeAsync(buf, s);
  if (iters_out) *iters_out = it;
  if (relres_out) *relres_out = rel;
  return rc;
}
