// bem_batch.cu -- many independent scatterers (meshes and wavenumbers) behind
// one handle, applied by one CUDA graph.
//
// Every problem keeps its own octree, operators and workspaces (a sub-handle
// built by bem_setup).  The batch apply stages the caller's concatenated
// densities into a fixed internal buffer, replays a CUDA graph that holds the
// applies of all problems, spread round-robin over BEM_BATCH_STREAMS forked
// streams so that small problems run concurrently, and scatters the results
// back.  One graph is captured per (nrhs, dtype, flags) on first use.
#include <algorithm>
#include <map>
#include <vector>

#include "bem_common.cuh"

#define BEM_BATCH_STREAMS 64

struct bem_batch {
  std::vector<bem_handle*> h;
  std::vector<int64_t> off;  // first column of every problem in the concatenated layout
  int64_t ntot = 0;
  int nrhs_max = 0;
  int device = 0;
  double* sx = nullptr;  // staging [sum_b nrhs_max * N_b] complex double, per-problem blocks
  double* sy = nullptr;
  double* sz = nullptr;
  cudaStream_t cs = nullptr;
  cudaStream_t fork[BEM_BATCH_STREAMS] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[BEM_BATCH_STREAMS] = {};
  std::map<int, cudaGraphExec_t> graphs;  // key: nrhs | half << 20
  int64_t* doff = nullptr;                // device copy of `off`
  std::vector<void*> allocs;
};

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// caller layout [nrhs][ntot] <-> staging blocks [problem][nrhs][N_b]
template <typename R>
__global__ void k_batch_gather(int64_t ntot, int nrhs, int nprob, const int64_t* __restrict__ off,
                               const R* __restrict__ in, double* __restrict__ stage) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ntot) return;
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {  // problem owning column c
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= c)
      lo = mid;
    else
      hi = mid - 1;
  }
  int64_t nb = off[lo + 1] - off[lo], j = c - off[lo];
  double* blk = stage + 2 * nrhs * off[lo];
  for (int r = 0; r < nrhs; ++r) {
    blk[2 * (r * nb + j)] = (double)in[2 * (r * ntot + c)];
    blk[2 * (r * nb + j) + 1] = (double)in[2 * (r * ntot + c) + 1];
  }
}

template <typename R>
__global__ void k_batch_scatter(int64_t ntot, int nrhs, int nprob, const int64_t* __restrict__ off,
                                const double* __restrict__ stage, R* __restrict__ out) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ntot) return;
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= c)
      lo = mid;
    else
      hi = mid - 1;
  }
  int64_t nb = off[lo + 1] - off[lo], j = c - off[lo];
  const double* blk = stage + 2 * nrhs * off[lo];
  for (int r = 0; r < nrhs; ++r) {
    out[2 * (r * ntot + c)] = (R)blk[2 * (r * nb + j)];
    out[2 * (r * ntot + c) + 1] = (R)blk[2 * (r * nb + j) + 1];
  }
}

static void free_batch(bem_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  for (auto* h : b->h) bem_destroy(h);
  for (void* p : b->allocs) cudaFree(p);
  for (int i = 0; i < BEM_BATCH_STREAMS; ++i) {
    if (b->fork[i]) cudaStreamDestroy(b->fork[i]);
    if (b->ev_join[i]) cudaEventDestroy(b->ev_join[i]);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->cs) cudaStreamDestroy(b->cs);
  delete b;
}

extern "C" int bem_destroy_batch(bem_batch* b) {
  bem_set_error("");
  free_batch(b);
  return BEM_OK;
}

// opt_stride 0: every problem takes opts[0] (nullable); 1: problem i takes opts[i]
static int setup_batch(const bem_mesh* meshes, const double* ks, int count, int p, double eps,
                       const bem_options* opts, int opt_stride, void* stream, bem_batch** out) {
  bem_set_error("");
  if (!out) return bem_fail(BEM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!meshes || !ks || count < 1) return bem_fail(BEM_ERR_INVALID_ARG, "need count >= 1 meshes and wavenumbers");
  if (opt_stride && !opts) return bem_fail(BEM_ERR_INVALID_ARG, "opts is NULL");
  bem_batch* b = new bem_batch();
  cudaGetDevice(&b->device);
  b->off.push_back(0);
  for (int i = 0; i < count; ++i) {
    bem_handle* h = nullptr;
    int rc = bem_setup(&meshes[i], ks[i], p, eps, opts ? opts + (size_t)i * opt_stride : nullptr, stream, &h);
    if (rc == BEM_OK && i > 0 && h->nrhs_max != b->h[0]->nrhs_max) {
      bem_destroy(h);
      rc = bem_fail(BEM_ERR_INVALID_ARG, "every problem must use the same max_nrhs");
    }
    if (rc != BEM_OK) {
      std::string m = "problem " + std::to_string(i) + ": " + bem_last_error();
      free_batch(b);
      return bem_fail(rc, m);
    }
    b->h.push_back(h);
    b->off.push_back(b->off.back() + h->nt);
  }
  b->ntot = b->off.back();
  b->nrhs_max = b->h[0]->nrhs_max;
  size_t n = 2 * (size_t)b->ntot * b->nrhs_max;
  cudaError_t e = cudaSuccess;
  for (double** pp : {&b->sx, &b->sy, &b->sz}) {
    e = cudaMalloc((void**)pp, n * sizeof(double));
    if (e != cudaSuccess) break;
    b->allocs.push_back(*pp);
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->doff, b->off.size() * sizeof(int64_t));
  if (e == cudaSuccess) {
    b->allocs.push_back(b->doff);
    e = cudaMemcpy(b->doff, b->off.data(), b->off.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking);
  for (int i = 0; i < BEM_BATCH_STREAMS && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&b->fork[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    std::string m = std::string("batch workspace: ") + cudaGetErrorString(e);
    free_batch(b);
    return bem_fail(e == cudaErrorMemoryAllocation ? BEM_ERR_OOM : BEM_ERR_CUDA, m);
  }
  *out = b;
  return BEM_OK;
}

extern "C" int bem_setup_batch(const bem_mesh* meshes, const double* ks, int count, int p, double eps,
                               const bem_options* opt, void* stream, bem_batch** out) {
  return setup_batch(meshes, ks, count, p, eps, opt, 0, stream, out);
}

extern "C" int bem_setup_batch_each(const bem_mesh* meshes, const double* ks, int count, int p, double eps,
                                    const bem_options* opts, void* stream, bem_batch** out) {
  return setup_batch(meshes, ks, count, p, eps, opts, 1, stream, out);
}

// the applies of all problems (staging buffers in, staging buffer out),
// forked over the batch's streams and joined back into `s`; the stage timers
// (events) stay off, so that the work can be captured
static int issue_batch(bem_batch* b, int nrhs, int half, cudaStream_t s) {
  int rc = BEM_OK;
  const int ns = std::min<int>(BEM_BATCH_STREAMS, (int)b->h.size());  // streams in use
  BEM_CUDA(cudaEventRecord(b->ev_fork, s));
  for (int i = 0; i < ns; ++i) BEM_CUDA(cudaStreamWaitEvent(b->fork[i], b->ev_fork, 0));
  for (size_t p = 0; p < b->h.size() && rc == BEM_OK; ++p) {
    bem_handle* h = b->h[p];
    cudaStream_t fs = b->fork[p % ns];
    const double* x = b->sx + 2 * nrhs * b->off[p];
    const double* y = b->sy + 2 * nrhs * b->off[p];
    double* z = b->sz + 2 * nrhs * b->off[p];
    const int prof = h->prof_on;
    h->prof_on = 0;
    rc = bem_prologue(h, nrhs, BEM_C128, x, y, fs);
    if (rc == BEM_OK) rc = bem_apply_sorted(h, nrhs, fs);
    if (rc == BEM_OK) rc = bem_epilogue(h, nrhs, BEM_C128, x, z, half, fs);
    h->prof_on = prof;
  }
  // join every forked stream, also after a failure, so that no stream is left
  // waiting outside a capture that ends
  for (int i = 0; i < ns; ++i) {
    cudaError_t e = cudaEventRecord(b->ev_join[i], b->fork[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev_join[i], 0);
    if (e != cudaSuccess && rc == BEM_OK) rc = bem_fail(BEM_ERR_CUDA, std::string("batch join: ") + cudaGetErrorString(e));
  }
  return rc;
}

// capture the applies of all problems into an executable graph
static int capture(bem_batch* b, int nrhs, int half, cudaGraphExec_t* exec) {
  cudaStream_t s = b->cs;
  BEM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  int rc = issue_batch(b, nrhs, half, s);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (rc != BEM_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return bem_fail(BEM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bem_fail(BEM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return BEM_OK;
}

extern "C" int bem_apply_batch(bem_batch* b, int nrhs, int dtype, const void* x, const void* y, void* z, int flags,
                               void* stream) {
  bem_set_error("");
  if (!b) return bem_fail(BEM_ERR_INVALID_ARG, "batch is NULL");
  if (nrhs < 1 || nrhs > b->nrhs_max) return bem_fail(BEM_ERR_INVALID_ARG, "nrhs out of [1, max_nrhs]");
  if (dtype != BEM_C64 && dtype != BEM_C128) return bem_fail(BEM_ERR_INVALID_ARG, "dtype must be BEM_C64 or BEM_C128");
  if (flags & ~BEM_APPLY_NO_HALF) return bem_fail(BEM_ERR_INVALID_ARG, "flags: only BEM_APPLY_NO_HALF");
  if (!z || (!x && !y)) return bem_fail(BEM_ERR_INVALID_ARG, "z and at least one of x, y are required");
  cudaStream_t s = (cudaStream_t)stream;
  int half = (flags & BEM_APPLY_NO_HALF) ? 0 : 1;
  int key = nrhs | (half << 20);
  auto it = b->graphs.find(key);
  if (it == b->graphs.end()) {
    cudaGraphExec_t ex = nullptr;
    BEM_TRY(capture(b, nrhs, half, &ex));
    it = b->graphs.emplace(key, ex).first;
  }
  const int64_t* doff = b->doff;
  int np = (int)b->h.size();
  unsigned g = nblk(b->ntot, 256);
  size_t bytes = 2 * (size_t)b->ntot * nrhs * sizeof(double);
  if (dtype == BEM_C128) {
    if (x) k_batch_gather<double><<<g, 256, 0, s>>>(b->ntot, nrhs, np, doff, (const double*)x, b->sx);
    else BEM_CUDA(cudaMemsetAsync(b->sx, 0, bytes, s));
    if (y) k_batch_gather<double><<<g, 256, 0, s>>>(b->ntot, nrhs, np, doff, (const double*)y, b->sy);
    else BEM_CUDA(cudaMemsetAsync(b->sy, 0, bytes, s));
  } else {
    if (x) k_batch_gather<float><<<g, 256, 0, s>>>(b->ntot, nrhs, np, doff, (const float*)x, b->sx);
    else BEM_CUDA(cudaMemsetAsync(b->sx, 0, bytes, s));
    if (y) k_batch_gather<float><<<g, 256, 0, s>>>(b->ntot, nrhs, np, doff, (const float*)y, b->sy);
    else BEM_CUDA(cudaMemsetAsync(b->sy, 0, bytes, s));
  }
  BEM_CUDA(cudaGetLastError());
  BEM_CUDA(cudaGraphLaunch(it->second, s));
  if (dtype == BEM_C128)
    k_batch_scatter<double><<<g, 256, 0, s>>>(b->ntot, nrhs, np, doff, b->sz, (double*)z);
  else
    k_batch_scatter<float><<<g, 256, 0, s>>>(b->ntot, nrhs, np, doff, b->sz, (float*)z);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

extern "C" int bem_batch_info(bem_batch* b, int problem, int key, int64_t* value) {
  bem_set_error("");
  if (!b || !value) return bem_fail(BEM_ERR_INVALID_ARG, "NULL argument");
  if (problem == -1) {
    if (key == 0) {
      *value = b->ntot;
      return BEM_OK;
    }
    if (key == 1) {
      *value = (int64_t)b->h.size();
      return BEM_OK;
    }
    return bem_fail(BEM_ERR_INVALID_ARG, "unknown batch key");
  }
  if (problem < 0 || problem >= (int)b->h.size()) return bem_fail(BEM_ERR_INVALID_ARG, "problem index out of range");
  return bem_info(b->h[problem], key, value);
}

// ------------------------------------------------------------ batch solve --
// GMRES for every problem and right-hand side of the batch at once: column
// (r, p) is problem p's segment of right-hand side r in the caller's
// [nrhs][ntot] layout, and each iteration is one batch apply of (1/2 I - D):
// captured into the solver's cycle graph, or graph-replayed from the host
// loop.  Columns converge independently (each has its own Krylov space).
namespace {
struct BatchOp {
  bem_batch* b;
  int nrhs;
};
int batch_apply(void* ctx, const double* in, double* out, cudaStream_t s) {
  BatchOp* o = (BatchOp*)ctx;
  return bem_apply_batch(o->b, o->nrhs, BEM_C128, in, nullptr, out, 0, (void*)s);
}
// the same work issued directly into `s` (for capture into a solver graph)
int batch_apply_capture(void* ctx, const double* in, double* out, cudaStream_t s) {
  BatchOp* o = (BatchOp*)ctx;
  bem_batch* b = o->b;
  const int np = (int)b->h.size();
  const unsigned g = nblk(b->ntot, 256);
  k_batch_gather<double><<<g, 256, 0, s>>>(b->ntot, o->nrhs, np, b->doff, in, b->sx);
  BEM_CUDA(cudaMemsetAsync(b->sy, 0, 2 * (size_t)b->ntot * o->nrhs * sizeof(double), s));
  BEM_TRY(issue_batch(b, o->nrhs, 1, s));
  k_batch_scatter<double><<<g, 256, 0, s>>>(b->ntot, o->nrhs, np, b->doff, b->sz, out);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}
}  // namespace

extern "C" int bem_gmres_solve_batch(bem_batch* b, int nrhs, int dtype, const void* rhs, void* x, double tol,
                                     int max_iter, int restart, int flags, int* iters_out, double* relres_out,
                                     void* stream) {
  bem_set_error("");
  if (!b) return bem_fail(BEM_ERR_INVALID_ARG, "batch is NULL");
  if (nrhs < 1 || nrhs > b->nrhs_max) return bem_fail(BEM_ERR_INVALID_ARG, "nrhs out of [1, max_nrhs]");
  if (dtype != BEM_C64 && dtype != BEM_C128) return bem_fail(BEM_ERR_INVALID_ARG, "dtype must be BEM_C64 or BEM_C128");
  if (!rhs || !x) return bem_fail(BEM_ERR_INVALID_ARG, "rhs and x are required");
  if (!(tol > 0.0) || max_iter < 1 || restart < 1)
    return bem_fail(BEM_ERR_INVALID_ARG, "tol must be > 0, max_iter and restart >= 1");
  if (flags & ~(BEM_GMRES_USE_X0 | BEM_GMRES_HOST_LOOP | BEM_GMRES_GRAPH_ONLY))
    return bem_fail(BEM_ERR_INVALID_ARG, "flags: BEM_GMRES_USE_X0 | BEM_GMRES_HOST_LOOP | BEM_GMRES_GRAPH_ONLY");
  const int np = (int)b->h.size();
  const int ncol = nrhs * np;
  std::vector<int64_t> off(ncol), len(ncol);
  for (int r = 0; r < nrhs; ++r)
    for (int p = 0; p < np; ++p) {
      off[r * np + p] = (int64_t)r * b->ntot + b->off[p];
      len[r * np + p] = b->off[p + 1] - b->off[p];
    }
  BatchOp ctx{b, nrhs};
  return bem_gmres_core(batch_apply, batch_apply_capture, &ctx, ncol, (int64_t)nrhs * b->ntot, off.data(), len.data(), dtype, rhs, x, tol,
                        max_iter, restart, flags, iters_out, relres_out, (cudaStream_t)stream);
}
