// bem_fem.cu -- the elastic half of Section 2.3's coupled solver on the GPU:
// P1 tetrahedra of the body Omega^c, K - rho_s omega^2 M assembled and
// factorised once (step 1 of the paper's algorithm), and the coupling map of
// Eq. (GMRES) applied in stream order (steps 2(a), 2(b)):
//   y = C x = rho_f omega^2 Avg (K - rho_s omega^2 M)^{-1} (-N x),
// N[(a,i), j] = n_ji A_j / 3 (the load of the piecewise constant pressure,
// with the traction t = -p n of the boundary condition), Avg[j, (a,i)] =
// n_ji / 3 (the element mean of u.n that the single layer takes as density).
//
// Element matrices (one thread per tetrahedron, FP64):
//   K_e[(a,i),(b,k)] = V (lambda g_ai g_bk + mu g_ak g_bi + mu delta_ik g_a.g_b),
//   M_e[(a,i),(b,k)] = delta_ik V (1 + delta_ab) / 20,
// g_a the constant gradient of corner a's P1 function, scattered by FP64
// atomic adds into a dense column-major matrix of order n = 3 n_nodes.
//
// The factor is a dense LU with partial pivoting (the paper uses a
// multifrontal sparse solver): right-looking, one column per step, a
// single-block kernel for the pivot search, the row swap and the column
// scale, then a rank-1 update of the trailing block.  The update moves 16
// bytes per multiply-add, so the factor is bound by HBM, where GB300's low
// FP64 rate does not matter; it costs n^3 / 3 multiply-adds.  Solves apply
// the row permutation, then forward and back substitution by blocks of 64
// rows: one warp per right-hand side column solves the diagonal block, and
// a grid kernel updates the rows below (above).
#include <cstring>
#include <vector>

#include "bem_common.cuh"

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

struct bem_fem {
  int device = 0;
  int64_t nn = 0, ntet = 0, ntri = 0, n = 0;  // n = 3 nn degrees of freedom
  double lam = 0, mu = 0, rho_s = 0, rho_f = 0, omega = 0;
  double* A = nullptr;      // [n][n] column-major; after setup L (unit lower) and U in place
  double* A0 = nullptr;     // the assembled matrix, kept with BEM_FEM_KEEP_MATRIX
  int* piv = nullptr;       // [n] the row swapped with row k at step k
  int* perm = nullptr;      // [n] (P b)[i] = b[perm[i]]
  double* dinv = nullptr;   // [n / FEM_SUB blocks][2][FEM_SUB][FEM_SUB]: inverses of L's and U's diagonal blocks
  int* tri = nullptr;       // [ntri][3]
  double* tn = nullptr;     // [ntri][4]: unit normal, area
  double* work = nullptr;   // [2 cap][n] real right-hand sides
  int cap = 0;              // complex right-hand sides that fit in work
  int* d_err = nullptr;     // device error word (singular pivot)
  int singular = 0;         // first zero pivot + 1, 0 if none
  const void* cx = nullptr;  // buffers bound for bem_fem_coupling
  void* cy = nullptr;
  int64_t bytes = 0;
};

#define FEM_SUB 64  // rows per block of the triangular solves

// ---------------------------------------------------------------- assembly --
__global__ void k_fem_assemble(int64_t ntet, const double* __restrict__ X, const int* __restrict__ tets, double lam,
                               double mu, double shift, int64_t n, double* __restrict__ A, int* __restrict__ err) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= ntet) return;
  int nd[4];
  double P[4][3];
  for (int a = 0; a < 4; ++a) {
    nd[a] = tets[4 * e + a];
    for (int d = 0; d < 3; ++d) P[a][d] = X[3 * (int64_t)nd[a] + d];
  }
  // J = [X1 - X0 | X2 - X0 | X3 - X0]; the rows of J^{-1} are the gradients of
  // the barycentric coordinates of corners 1..3
  double J[3][3];
  for (int d = 0; d < 3; ++d)
    for (int c = 0; c < 3; ++c) J[d][c] = P[c + 1][d] - P[0][d];
  const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  if (!(fabs(det) > 0.0)) {
    atomicOr(err, 1);
    return;
  }
  const double id = 1.0 / det;
  double g[4][3];
  // inverse = adjugate / det; row r of J^{-1} is g[r + 1]
  g[1][0] = c00 * id;
  g[2][0] = c01 * id;
  g[3][0] = c02 * id;
  g[1][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
  g[2][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
  g[3][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
  g[1][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
  g[2][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
  g[3][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
  for (int d = 0; d < 3; ++d) g[0][d] = -(g[1][d] + g[2][d] + g[3][d]);
  const double V = fabs(det) / 6.0;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      const double gg = g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2];
      const double me = V * (a == b ? 2.0 : 1.0) / 20.0;
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) {
          double v = V * (lam * g[a][i] * g[b][k] + mu * g[a][k] * g[b][i]);
          if (i == k) v += V * mu * gg - shift * me;
          const int64_t row = 3 * (int64_t)nd[a] + i, col = 3 * (int64_t)nd[b] + k;
          atomicAdd(&A[col * n + row], v);
        }
    }
}

// ----------------------------------------------------------------------- LU --
// Step k, one block: the pivot p = argmax_{i >= k} |A[i][k]| (the smallest
// index among equal magnitudes), rows k and p swapped across every column,
// then A[i][k] /= A[k][k] for i > k.  A zero column records step k + 1 in
// err (the first one wins) and leaves the column as it is.
__global__ void __launch_bounds__(1024) k_fem_pivot(int64_t n, int64_t k, double* __restrict__ A, int* __restrict__ piv,
                                                    int* __restrict__ err) {
  __shared__ double s_v[1024];
  __shared__ int64_t s_i[1024];
  double best = -1.0;
  int64_t bi = k;
  for (int64_t i = k + threadIdx.x; i < n; i += blockDim.x) {
    const double v = fabs(A[k * n + i]);
    if (v > best) {
      best = v;
      bi = i;
    }
  }
  s_v[threadIdx.x] = best;
  s_i[threadIdx.x] = bi;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      const double v = s_v[threadIdx.x + st];
      const int64_t i = s_i[threadIdx.x + st];
      if (v > s_v[threadIdx.x] || (v == s_v[threadIdx.x] && i < s_i[threadIdx.x])) {
        s_v[threadIdx.x] = v;
        s_i[threadIdx.x] = i;
      }
    }
    __syncthreads();
  }
  const int64_t p = s_i[0];
  const bool zero = !(s_v[0] > 0.0);
  if (threadIdx.x == 0) {
    piv[k] = (int)p;
    if (zero) atomicCAS(err, 0, (int)(k + 1));
  }
  if (p != k)
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      const double t = A[j * n + k];
      A[j * n + k] = A[j * n + p];
      A[j * n + p] = t;
    }
  __syncthreads();
  if (zero) return;
  const double inv = 1.0 / A[k * n + k];
  for (int64_t i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[k * n + i] *= inv;
}

// Step k's rank-1 update: A[i][j] -= A[i][k] A[k][j] for i, j > k.  Blocks of
// 32 x 32 (threads 32 x 8, four columns each); x over rows, so a warp reads a
// column segment.
__global__ void __launch_bounds__(256) k_fem_update(int64_t n, int64_t k, double* __restrict__ A) {
  const int64_t i = k + 1 + blockIdx.x * 32 + threadIdx.x;
  const int64_t j0 = k + 1 + blockIdx.y * 32 + threadIdx.y;
  if (i >= n) return;
  const double l = A[k * n + i];
  for (int c = 0; c < 4; ++c) {
    const int64_t j = j0 + 8 * c;
    if (j < n) A[j * n + i] -= l * A[j * n + k];
  }
}

// -------------------------------------------------------------- solves --
// Y [ncol][n]: (P b) gathered from B through perm
__global__ void k_fem_permute(int64_t n, int ncol, const int* __restrict__ perm, const double* __restrict__ B,
                              double* __restrict__ Y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t s = perm[i];
  for (int c = 0; c < ncol; ++c) Y[(int64_t)c * n + i] = B[(int64_t)c * n + s];
}

// Inverses of the diagonal blocks of L (unit lower) and U (upper), one block
// of FEM_SUB rows per CTA, after the factorisation: thread t solves for
// column t of the inverse by substitution (inv[r][t], row-major in Dinv).
__global__ void __launch_bounds__(FEM_SUB) k_fem_diag_inv(int64_t n, const double* __restrict__ A,
                                                          double* __restrict__ Dinv) {
  __shared__ double s_a[FEM_SUB][FEM_SUB + 1];  // [row][column]
  const int64_t k0 = blockIdx.x * (int64_t)FEM_SUB;
  const int nb = (int)min((int64_t)FEM_SUB, n - k0);
  for (int j = 0; j < nb; ++j)
    if (threadIdx.x < nb) s_a[threadIdx.x][j] = A[(k0 + j) * n + k0 + threadIdx.x];
  __syncthreads();
  const int t = threadIdx.x;
  double* Li = Dinv + (int64_t)blockIdx.x * 2 * FEM_SUB * FEM_SUB;
  double* Ui = Li + FEM_SUB * FEM_SUB;
  double col[FEM_SUB];
  // L x = e_t (unit diagonal)
  for (int r = 0; r < FEM_SUB; ++r) {
    double v = (r == t) ? 1.0 : 0.0;
    for (int j = 0; j < r; ++j) v -= (r < nb && j < nb) ? s_a[r][j] * col[j] : 0.0;
    col[r] = v;
  }
  for (int r = 0; r < FEM_SUB; ++r) Li[r * FEM_SUB + t] = (r < nb && t < nb) ? col[r] : 0.0;
  // U x = e_t
  for (int r = FEM_SUB - 1; r >= 0; --r) {
    double v = (r == t) ? 1.0 : 0.0;
    for (int j = r + 1; j < FEM_SUB; ++j) v -= (r < nb && j < nb) ? s_a[r][j] * col[j] : 0.0;
    col[r] = (r < nb) ? v / s_a[r][r] : 0.0;
  }
  for (int r = 0; r < FEM_SUB; ++r) Ui[r * FEM_SUB + t] = (r < nb && t < nb) ? col[r] : 0.0;
}

// One substitution step on the rows [k0, k0 + nb) (one launch per step):
// every CTA forms the step's solution s = Dinv_k y[k0 .. k0 + nb) of every
// column in shared memory, CTA 0 stores it in Out, and each CTA updates its 32
// rows of [r0, r1): In_i -= sum_j A[i][k0 + j] s_j.  In rows [k0, k0 + nb) are
// only read during the step, so no CTA waits for another.  The 8 warps of a
// CTA split the step's columns (warp w takes j = w, w + 8, ...): each load is a
// coalesced column segment; the partial sums of a row meet in shared memory.
__global__ void __launch_bounds__(256) k_fem_step(int64_t n, int64_t k0, int nb, int64_t r0, int64_t r1, int ncol,
                                                  const double* __restrict__ A, const double* __restrict__ Dk,
                                                  double* __restrict__ In, double* __restrict__ Out) {
  extern __shared__ double s_y[];  // [ncol][FEM_SUB] right-hand sides, [ncol][FEM_SUB] solutions, [8][32],
                                   // then Dk as [FEM_SUB][FEM_SUB + 1]
  double* s_s = s_y + ncol * FEM_SUB;
  double* s_p = s_s + ncol * FEM_SUB;
  double* s_d = s_p + 8 * 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // this CTA's rows of the step's columns first: their loads overlap the rest
  const int64_t i = r0 + blockIdx.x * (int64_t)32 + lane;
  const bool live = i < r1;
  double a[FEM_SUB / 8];
#pragma unroll
  for (int u = 0; u < FEM_SUB / 8; ++u) {
    const int j = w + 8 * u;
    a[u] = (live && j < nb) ? A[(k0 + j) * n + i] : 0.0;
  }
  for (int t = threadIdx.x; t < ncol * FEM_SUB; t += blockDim.x) {
    const int c = t / FEM_SUB, j = t % FEM_SUB;
    s_y[t] = j < nb ? In[(int64_t)c * n + k0 + j] : 0.0;
  }
  for (int t = threadIdx.x; t < FEM_SUB * FEM_SUB; t += blockDim.x)
    s_d[(t / FEM_SUB) * (FEM_SUB + 1) + t % FEM_SUB] = Dk[t];
  __syncthreads();
  // the step's solution from shared memory (rows of Dk at a stride of 65:
  // consecutive threads, consecutive rows, no bank conflicts)
  for (int o = threadIdx.x; o < ncol * FEM_SUB; o += blockDim.x) {
    const int c = o / FEM_SUB, r = o % FEM_SUB;
    const double* d = s_d + r * (FEM_SUB + 1);
    const double* y = s_y + c * FEM_SUB;
    double v = 0.0;
#pragma unroll 16
    for (int j = 0; j < FEM_SUB; ++j) v += d[j] * y[j];
    s_s[o] = v;
    if (blockIdx.x == 0 && r < nb) Out[(int64_t)c * n + k0 + r] = v;
  }
  __syncthreads();
  for (int c = 0; c < ncol; ++c) {
    double acc = 0.0;
#pragma unroll
    for (int u = 0; u < FEM_SUB / 8; ++u) acc += a[u] * s_s[c * FEM_SUB + w + 8 * u];
    s_p[w * 32 + lane] = acc;
    __syncthreads();
    if (w == 0 && live) {
      double t = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) t += s_p[q * 32 + lane];
      In[(int64_t)c * n + i] -= t;
    }
    __syncthreads();
  }
}

// the load of the pressures x (complex [nrhs][ntri], dtype Rin) into real
// columns B[2 r] (real part) and B[2 r + 1] (imaginary part): -N x
template <typename Rin>
__global__ void k_fem_load(int64_t ntri, int nrhs, int64_t n, const int* __restrict__ tri,
                           const double* __restrict__ tn, const Rin* __restrict__ x, double* __restrict__ B) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= ntri) return;
  const double w = tn[4 * j + 3] / 3.0;
  for (int r = 0; r < nrhs; ++r) {
    const double xr = (double)x[2 * ((int64_t)r * ntri + j)], xi = (double)x[2 * ((int64_t)r * ntri + j) + 1];
    for (int a = 0; a < 3; ++a) {
      const int64_t node = tri[3 * j + a];
      for (int d = 0; d < 3; ++d) {
        const double f = -w * tn[4 * j + d];
        atomicAdd(&B[(int64_t)(2 * r) * n + 3 * node + d], f * xr);
        atomicAdd(&B[(int64_t)(2 * r + 1) * n + 3 * node + d], f * xi);
      }
    }
  }
}

// y_j = beta n_j . (u_a + u_b + u_c) / 3 from the real columns U[2 r], U[2 r + 1]
template <typename Rout>
__global__ void k_fem_avg(int64_t ntri, int nrhs, int64_t n, const int* __restrict__ tri,
                          const double* __restrict__ tn, const double* __restrict__ U, double beta,
                          Rout* __restrict__ y) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= ntri) return;
  for (int r = 0; r < nrhs; ++r) {
    double sr = 0.0, si = 0.0;
    for (int a = 0; a < 3; ++a) {
      const int64_t node = tri[3 * j + a];
      for (int d = 0; d < 3; ++d) {
        sr += tn[4 * j + d] * U[(int64_t)(2 * r) * n + 3 * node + d];
        si += tn[4 * j + d] * U[(int64_t)(2 * r + 1) * n + 3 * node + d];
      }
    }
    y[2 * ((int64_t)r * ntri + j)] = (Rout)(beta * sr / 3.0);
    y[2 * ((int64_t)r * ntri + j) + 1] = (Rout)(beta * si / 3.0);
  }
}

// ------------------------------------------------------------------- host --
static void fem_free(bem_fem* f) {
  if (!f) return;
  for (void* p : {(void*)f->A, (void*)f->A0, (void*)f->piv, (void*)f->perm, (void*)f->dinv, (void*)f->tri,
                  (void*)f->tn, (void*)f->work, (void*)f->d_err})
    if (p) cudaFree(p);
  delete f;
}

// forward and back substitution of the permuted columns Y [ncol][n]; X
// [ncol][n] is scratch; the solution ends in Y.  One launch per block of
// FEM_SUB rows and direction.
static int fem_substitute(bem_fem* f, int ncol, double* Y, double* X, cudaStream_t s) {
  const int64_t n = f->n, nbk = (n + FEM_SUB - 1) / FEM_SUB;
  const size_t sh = sizeof(double) * (2 * (size_t)ncol * FEM_SUB + 8 * 32 + FEM_SUB * (FEM_SUB + 1));
  for (int64_t b = 0; b < nbk; ++b) {  // L z = P y: Y -> X
    const int64_t k0 = b * FEM_SUB, r0 = k0 + FEM_SUB;
    const int nb = (int)std::min<int64_t>(FEM_SUB, n - k0);
    const unsigned g = r0 < n ? nblk(n - r0, 32) : 1;
    k_fem_step<<<g, 256, sh, s>>>(n, k0, nb, r0, n, ncol, f->A, f->dinv + b * 2 * FEM_SUB * FEM_SUB, Y, X);
  }
  for (int64_t b = nbk - 1; b >= 0; --b) {  // U x = z: X -> Y
    const int64_t k0 = b * FEM_SUB;
    const int nb = (int)std::min<int64_t>(FEM_SUB, n - k0);
    const unsigned g = k0 > 0 ? nblk(k0, 32) : 1;
    k_fem_step<<<g, 256, sh, s>>>(n, k0, nb, 0, k0, ncol, f->A, f->dinv + (b * 2 + 1) * FEM_SUB * FEM_SUB, X, Y);
  }
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

static int fem_reserve(bem_fem* f, int nrhs) {
  if (nrhs <= f->cap) return BEM_OK;
  if (f->work) {
    BEM_CUDA(cudaFree(f->work));
    f->bytes -= (int64_t)sizeof(double) * 4 * f->cap * f->n;
    f->work = nullptr;
    f->cap = 0;
  }
  // two real columns per complex right-hand side, twice (load and solution)
  BEM_CUDA(cudaMalloc((void**)&f->work, sizeof(double) * 4 * (size_t)nrhs * f->n));
  f->cap = nrhs;
  f->bytes += (int64_t)sizeof(double) * 4 * nrhs * f->n;
  return BEM_OK;
}

extern "C" {

int bem_fem_setup(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets, const int32_t* tris,
                  int64_t n_tris, double lambda, double mu, double rho_s, double rho_f, double omega, int flags,
                  void* stream, bem_fem** out) {
  bem_set_error("");
  if (!out) return bem_fail(BEM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!nodes || !tets || !tris) return bem_fail(BEM_ERR_INVALID_ARG, "nodes, tets and tris are required");
  if (n_nodes < 4 || n_tets < 1 || n_tris < 1) return bem_fail(BEM_ERR_INVALID_ARG, "empty body");
  if (3 * n_nodes > 60000) return bem_fail(BEM_ERR_INVALID_ARG, "more than 60,000 degrees of freedom");
  if (!(mu > 0.0) || !(lambda > -2.0 * mu / 3.0) || !(rho_s >= 0.0) || !std::isfinite(rho_f) ||
      !std::isfinite(omega) || !std::isfinite(lambda))
    return bem_fail(BEM_ERR_INVALID_ARG, "material parameters out of range");
  for (int64_t i = 0; i < 4 * n_tets; ++i)
    if (tets[i] < 0 || tets[i] >= n_nodes) return bem_fail(BEM_ERR_INVALID_ARG, "tetrahedron node out of range");
  for (int64_t i = 0; i < 3 * n_tris; ++i)
    if (tris[i] < 0 || tris[i] >= n_nodes) return bem_fail(BEM_ERR_INVALID_ARG, "triangle node out of range");
  cudaStream_t s = (cudaStream_t)stream;
  bem_fem* f = new bem_fem();
  cudaGetDevice(&f->device);
  f->nn = n_nodes;
  f->ntet = n_tets;
  f->ntri = n_tris;
  f->n = 3 * n_nodes;
  f->lam = lambda;
  f->mu = mu;
  f->rho_s = rho_s;
  f->rho_f = rho_f;
  f->omega = omega;
  const int64_t n = f->n;
  // triangle normals and areas on the host (FP64)
  std::vector<double> tn(4 * n_tris);
  for (int64_t j = 0; j < n_tris; ++j) {
    const double* a = nodes + 3 * (int64_t)tris[3 * j];
    const double* b = nodes + 3 * (int64_t)tris[3 * j + 1];
    const double* c = nodes + 3 * (int64_t)tris[3 * j + 2];
    const double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    const double cr[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
    const double l = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    if (!(l > 0.0)) {
      fem_free(f);
      return bem_fail(BEM_ERR_INVALID_ARG, "degenerate boundary triangle");
    }
    for (int d = 0; d < 3; ++d) tn[4 * j + d] = cr[d] / l;
    tn[4 * j + 3] = 0.5 * l;
  }
  double* dX = nullptr;
  int* dT = nullptr;
  int rc = BEM_OK;
  auto cu = [&](cudaError_t e) {
    if (rc == BEM_OK && e != cudaSuccess)
      rc = bem_fail(e == cudaErrorMemoryAllocation ? BEM_ERR_OOM : BEM_ERR_CUDA, cudaGetErrorString(e));
    return rc != BEM_OK;
  };
  do {
    const size_t mat = sizeof(double) * (size_t)n * n;
    if (cu(cudaMalloc((void**)&f->A, mat))) break;
    f->bytes += (int64_t)mat;
    if (flags & BEM_FEM_KEEP_MATRIX) {
      if (cu(cudaMalloc((void**)&f->A0, mat))) break;
      f->bytes += (int64_t)mat;
    }
    if (cu(cudaMalloc((void**)&f->piv, sizeof(int) * n))) break;
    if (cu(cudaMalloc((void**)&f->perm, sizeof(int) * n))) break;
    const int64_t nbk = (n + FEM_SUB - 1) / FEM_SUB;
    if (cu(cudaMalloc((void**)&f->dinv, sizeof(double) * 2 * FEM_SUB * FEM_SUB * nbk))) break;
    f->bytes += (int64_t)sizeof(double) * 2 * FEM_SUB * FEM_SUB * nbk;
    if (cu(cudaMalloc((void**)&f->tri, sizeof(int) * 3 * n_tris))) break;
    if (cu(cudaMalloc((void**)&f->tn, sizeof(double) * 4 * n_tris))) break;
    if (cu(cudaMalloc((void**)&f->d_err, sizeof(int)))) break;
    if (cu(cudaMallocAsync((void**)&dX, sizeof(double) * 3 * n_nodes, s))) break;
    if (cu(cudaMallocAsync((void**)&dT, sizeof(int) * 4 * n_tets, s))) break;
    if (cu(cudaMemcpyAsync(dX, nodes, sizeof(double) * 3 * n_nodes, cudaMemcpyHostToDevice, s))) break;
    if (cu(cudaMemcpyAsync(dT, tets, sizeof(int) * 4 * n_tets, cudaMemcpyHostToDevice, s))) break;
    if (cu(cudaMemcpyAsync(f->tri, tris, sizeof(int) * 3 * n_tris, cudaMemcpyHostToDevice, s))) break;
    if (cu(cudaMemcpyAsync(f->tn, tn.data(), sizeof(double) * 4 * n_tris, cudaMemcpyHostToDevice, s))) break;
    if (cu(cudaMemsetAsync(f->d_err, 0, sizeof(int), s))) break;
    if (cu(cudaMemsetAsync(f->A, 0, mat, s))) break;
    // step 1: assemble K - rho_s omega^2 M ...
    k_fem_assemble<<<nblk(n_tets, 128), 128, 0, s>>>(n_tets, dX, dT, lambda, mu, rho_s * omega * omega, n, f->A,
                                                     f->d_err);
    if (cu(cudaGetLastError())) break;
    int h_err = 0;
    if (cu(cudaMemcpyAsync(&h_err, f->d_err, sizeof(int), cudaMemcpyDeviceToHost, s))) break;
    if (cu(cudaStreamSynchronize(s))) break;
    if (h_err) {
      rc = bem_fail(BEM_ERR_INVALID_ARG, "degenerate tetrahedron");
      break;
    }
    if (f->A0 && cu(cudaMemcpyAsync(f->A0, f->A, mat, cudaMemcpyDeviceToDevice, s))) break;
    // ... and factorise it
    for (int64_t k = 0; k < n && rc == BEM_OK; ++k) {
      k_fem_pivot<<<1, 1024, 0, s>>>(n, k, f->A, f->piv, f->d_err);
      const int64_t m = n - k - 1;
      if (m > 0) k_fem_update<<<dim3(nblk(m, 32), nblk(m, 32)), dim3(32, 8), 0, s>>>(n, k, f->A);
      if ((k & 1023) == 0) cu(cudaGetLastError());
    }
    if (cu(cudaGetLastError())) break;
    k_fem_diag_inv<<<(unsigned)nbk, FEM_SUB, 0, s>>>(n, f->A, f->dinv);
    // the substitution steps hold two [64 columns][FEM_SUB] tiles at most and a diagonal block
    if (cu(cudaFuncSetAttribute(k_fem_step, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(double) * (2 * 64 * FEM_SUB + 8 * 32 + FEM_SUB * (FEM_SUB + 1))))))
      break;
    if (cu(cudaGetLastError())) break;
    std::vector<int> piv(n), perm(n);
    if (cu(cudaMemcpyAsync(piv.data(), f->piv, sizeof(int) * n, cudaMemcpyDeviceToHost, s))) break;
    if (cu(cudaMemcpyAsync(&h_err, f->d_err, sizeof(int), cudaMemcpyDeviceToHost, s))) break;
    if (cu(cudaStreamSynchronize(s))) break;
    f->singular = h_err;
    for (int64_t i = 0; i < n; ++i) perm[i] = (int)i;
    for (int64_t k = 0; k < n; ++k) std::swap(perm[k], perm[piv[k]]);
    if (cu(cudaMemcpyAsync(f->perm, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s))) break;
    if (cu(cudaStreamSynchronize(s))) break;
  } while (false);
  if (dX) cudaFreeAsync(dX, s);
  if (dT) cudaFreeAsync(dT, s);
  if (rc != BEM_OK) {
    cudaStreamSynchronize(s);
    fem_free(f);
    return rc;
  }
  if (f->singular) {
    fem_free(f);
    return bem_fail(BEM_ERR_INVALID_ARG, "K - rho_s omega^2 M is singular (omega^2 an eigenvalue of the body)");
  }
  *out = f;
  return BEM_OK;
}

int bem_fem_destroy(bem_fem* f) {
  bem_set_error("");
  fem_free(f);
  return BEM_OK;
}

int bem_fem_solve(bem_fem* f, int nrhs, const double* b, double* u, void* stream) {
  bem_set_error("");
  if (!f || !b || !u) return bem_fail(BEM_ERR_INVALID_ARG, "body, b and u are required");
  if (nrhs < 1 || nrhs > 64) return bem_fail(BEM_ERR_INVALID_ARG, "nrhs must be in [1, 64]");
  cudaStream_t s = (cudaStream_t)stream;
  BEM_TRY(fem_reserve(f, (nrhs + 1) / 2));
  double* tmp = f->work;  // the permuted copy, solved in place
  double* scr = f->work + (size_t)nrhs * f->n;
  k_fem_permute<<<nblk(f->n, 256), 256, 0, s>>>(f->n, nrhs, f->perm, b, tmp);
  BEM_TRY(fem_substitute(f, nrhs, tmp, scr, s));
  BEM_CUDA(cudaMemcpyAsync(u, tmp, sizeof(double) * (size_t)nrhs * f->n, cudaMemcpyDeviceToDevice, s));
  return BEM_OK;
}

int bem_fem_couple(bem_fem* f, int nrhs, int dtype, const void* x, void* y, void* stream) {
  bem_set_error("");
  if (!f || !x || !y) return bem_fail(BEM_ERR_INVALID_ARG, "body, x and y are required");
  if (nrhs < 1 || nrhs > 32) return bem_fail(BEM_ERR_INVALID_ARG, "nrhs must be in [1, 32]");
  if (dtype != BEM_C64 && dtype != BEM_C128) return bem_fail(BEM_ERR_INVALID_ARG, "dtype must be BEM_C64 or BEM_C128");
  cudaStream_t s = (cudaStream_t)stream;
  BEM_TRY(fem_reserve(f, nrhs));
  const int64_t n = f->n;
  const int ncol = 2 * nrhs;
  double* B = f->work;
  double* Y = f->work + (size_t)ncol * n;
  BEM_CUDA(cudaMemsetAsync(B, 0, sizeof(double) * (size_t)ncol * n, s));
  const unsigned gt = nblk(f->ntri, 128);
  if (dtype == BEM_C128)
    k_fem_load<double><<<gt, 128, 0, s>>>(f->ntri, nrhs, n, f->tri, f->tn, (const double*)x, B);
  else
    k_fem_load<float><<<gt, 128, 0, s>>>(f->ntri, nrhs, n, f->tri, f->tn, (const float*)x, B);
  k_fem_permute<<<nblk(n, 256), 256, 0, s>>>(n, ncol, f->perm, B, Y);
  BEM_TRY(fem_substitute(f, ncol, Y, B, s));
  const double beta = f->rho_f * f->omega * f->omega;
  if (dtype == BEM_C128)
    k_fem_avg<double><<<gt, 128, 0, s>>>(f->ntri, nrhs, n, f->tri, f->tn, Y, beta, (double*)y);
  else
    k_fem_avg<float><<<gt, 128, 0, s>>>(f->ntri, nrhs, n, f->tri, f->tn, Y, beta, (float*)y);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

int bem_fem_bind(bem_fem* f, const void* cx, void* cy) {
  bem_set_error("");
  if (!f) return bem_fail(BEM_ERR_INVALID_ARG, "body is NULL");
  f->cx = cx;
  f->cy = cy;
  return BEM_OK;
}

int bem_fem_coupling(void* ctx, int nrhs, void* stream) {
  bem_fem* f = (bem_fem*)ctx;
  if (!f || !f->cx || !f->cy) return bem_fail(BEM_ERR_INVALID_ARG, "no buffers bound (bem_fem_bind)");
  return bem_fem_couple(f, nrhs, BEM_C128, f->cx, f->cy, stream);
}

int bem_fem_matrix(bem_fem* f, double* out, void* stream) {
  bem_set_error("");
  if (!f || !out) return bem_fail(BEM_ERR_INVALID_ARG, "body and out are required");
  if (!f->A0) return bem_fail(BEM_ERR_UNSUPPORTED, "set up without BEM_FEM_KEEP_MATRIX");
  cudaStream_t s = (cudaStream_t)stream;
  BEM_CUDA(cudaMemcpyAsync(out, f->A0, sizeof(double) * (size_t)f->n * f->n, cudaMemcpyDefault, s));
  BEM_CUDA(cudaStreamSynchronize(s));
  return BEM_OK;
}

int bem_fem_info(bem_fem* f, int key, int64_t* value) {
  bem_set_error("");
  if (!f || !value) return bem_fail(BEM_ERR_INVALID_ARG, "body and value are required");
  switch (key) {
    case BEM_FEM_INFO_DOF: *value = f->n; return BEM_OK;
    case BEM_FEM_INFO_NODES: *value = f->nn; return BEM_OK;
    case BEM_FEM_INFO_TETS: *value = f->ntet; return BEM_OK;
    case BEM_FEM_INFO_TRIS: *value = f->ntri; return BEM_OK;
    case BEM_FEM_INFO_BYTES: *value = f->bytes; return BEM_OK;
    default: return bem_fail(BEM_ERR_INVALID_ARG, "unknown info key");
  }
}

}  // extern "C"
