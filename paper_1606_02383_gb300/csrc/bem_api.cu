// bem_api.cu -- the C ABI: argument checking, handle lifetime, orchestration.
#include <cmath>
#include <cstring>
#include <string>

#include "bem_common.cuh"

static thread_local std::string g_last_error;

void bem_set_error(const std::string& m) { g_last_error = m; }
int bem_fail(int code, const std::string& m) {
  g_last_error = m;
  return code;
}

bool bem_is_fmm(const bem_handle* h) {
  return h->mode == BEM_MODE_FMM_MIXED || h->mode == BEM_MODE_FMM_FP64 || h->mode == BEM_MODE_FMM_TF32;
}
bool bem_is_fp64(const bem_handle* h) { return h->mode == BEM_MODE_FMM_FP64 || h->mode == BEM_MODE_DIRECT_FP64; }

int bem_check_device_error(bem_handle* h, cudaStream_t s) {
  int flags = 0;
  BEM_CUDA(cudaMemcpyAsync(&flags, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  BEM_CUDA(cudaStreamSynchronize(s));
  if (flags == 0) return BEM_OK;
  BEM_CUDA(cudaMemsetAsync(h->d_err, 0, sizeof(int), s));
  if (flags & BEM_DEVERR_DEGENERATE) return bem_fail(BEM_ERR_DEGENERATE_MESH, "degenerate or invalid triangle");
  if (flags & BEM_DEVERR_TIMEOUT) return bem_fail(BEM_ERR_TIMEOUT, "a bounded device wait expired (tensor-core stage)");
  if (flags & BEM_DEVERR_OVERFLOW)
    return bem_fail(BEM_ERR_NUMERIC, "translation operator or expansion row not finite (order/frequency out of range)");
  return bem_fail(BEM_ERR_NUMERIC, "non-finite value detected on the device");
}

static cudaEvent_t ev_get(bem_handle* h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

int bem_prof_begin(bem_handle* h, cudaStream_t s) {
  if (!h->prof_on) return -1;
  ProfRec r;
  r.stage = -1;
  r.a = ev_get(h);
  r.b = ev_get(h);
  r.launches = 0;
  if (!r.a || !r.b) return -1;
  cudaEventRecord(r.a, s);
  h->prof.push_back(r);
  return (int)h->prof.size() - 1;
}

void bem_prof_end(bem_handle* h, int rec, int stage, int launches, cudaStream_t s) {
  h->launches_last_apply += launches;
  if (rec < 0) return;
  ProfRec& r = h->prof[rec];
  r.stage = stage;
  r.launches = launches;
  cudaEventRecord(r.b, s);
}

static void free_handle(bem_handle* h) {
  if (!h) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  for (auto& r : h->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  if (h->s_far) cudaStreamDestroy(h->s_far);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  cudaSetDevice(cur);
  delete h;
}

extern "C" {

const char* bem_last_error(void) { return g_last_error.c_str(); }

int bem_sync(bem_handle* h, void* stream) {
  bem_set_error("");
  if (!h) return bem_fail(BEM_ERR_INVALID_ARG, "handle is NULL");
  return bem_check_device_error(h, (cudaStream_t)stream);
}

int bem_set_wait_limit(bem_handle* h, long long clocks, int hold) {
  bem_set_error("");
  if (!h) return bem_fail(BEM_ERR_INVALID_ARG, "handle is NULL");
  h->tc_wait_limit = clocks > 0 ? clocks : (1LL << 31);
  h->tc_hold_first_copy = hold ? 1 : 0;
  return BEM_OK;
}

int bem_destroy(bem_handle* h) {
  g_last_error.clear();
  free_handle(h);
  return BEM_OK;
}

int bem_setup(const bem_mesh* mesh, double k, int p, double eps, const bem_options* opt, void* stream,
              bem_handle** out) {
  g_last_error.clear();
  if (!out) return bem_fail(BEM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!mesh || !mesh->vertices || !mesh->triangles) return bem_fail(BEM_ERR_INVALID_ARG, "mesh or its arrays NULL");
  if (mesh->n_triangles <= 0 || mesh->n_vertices < 3) return bem_fail(BEM_ERR_INVALID_ARG, "empty mesh");
  if (mesh->n_triangles > (int64_t)1 << 30) return bem_fail(BEM_ERR_INVALID_ARG, "more than 2^30 triangles");
  if (!(k > 0.0) || !std::isfinite(k)) return bem_fail(BEM_ERR_INVALID_ARG, "wavenumber must be finite and > 0");
  if (p < 0 || p > 60) return bem_fail(BEM_ERR_INVALID_ARG, "order p must be in [0, 60]");
  if (p == 0 && !(eps > 0.0 && eps < 1.0)) return bem_fail(BEM_ERR_INVALID_ARG, "eps must be in (0, 1)");
  bem_options o;
  memset(&o, 0, sizeof(o));
  o.mode = BEM_MODE_FMM_MIXED;
  o.leaf_target = 48;
  o.max_nrhs = 16;
  o.p_min = 4;
  o.p_max = 40;
  o.p2p_unit = 64;
  o.tc_kslice = 16;
  if (opt && opt->struct_size > 0) {
    size_t n = std::min((size_t)opt->struct_size, sizeof(o));
    memcpy(&o, opt, n);
    if (o.leaf_target <= 0) o.leaf_target = 48;
    if (o.max_nrhs <= 0) o.max_nrhs = 16;
    if (o.p_min <= 0) o.p_min = 4;
    if (o.p_max <= 0) o.p_max = 40;
    if (o.p2p_unit <= 0) o.p2p_unit = 64;
    if (o.tc_kslice <= 0) o.tc_kslice = 16;
  }
  if (o.mode < 0 || o.mode > 4) return bem_fail(BEM_ERR_INVALID_ARG, "unknown mode");
  if (o.max_nrhs > 1024) return bem_fail(BEM_ERR_INVALID_ARG, "max_nrhs above 1024");
  if (o.leaf_level > BEM_MAXLEV) return bem_fail(BEM_ERR_INVALID_ARG, "leaf_level above 10");
  if (o.leaf_level < -2) return bem_fail(BEM_ERR_INVALID_ARG, "leaf_level below -2");
  if (o.p_min > o.p_max || o.p_max > 60) return bem_fail(BEM_ERR_INVALID_ARG, "bad order bounds");
  if (o.p2p_unit != 16 && o.p2p_unit != 32 && o.p2p_unit != 64)
    return bem_fail(BEM_ERR_INVALID_ARG, "p2p_unit must be 16, 32 or 64");
  if (o.tc_kslice < 2 || o.tc_kslice > 16) return bem_fail(BEM_ERR_INVALID_ARG, "tc_kslice must be in [2, 16]");
  if (o.tc_pipeline < 0 || o.tc_pipeline > 4) return bem_fail(BEM_ERR_INVALID_ARG, "tc_pipeline must be in [0, 4]");
  if (o.p2p_ctas < 0 || o.p2p_ctas > 16) return bem_fail(BEM_ERR_INVALID_ARG, "p2p_ctas must be in [0, 16]");

  cudaStream_t s = (cudaStream_t)stream;
  bem_handle* h = new bem_handle();
  cudaGetDevice(&h->device);
  h->mode = o.mode;
  h->k = k;
  h->fixed_p = p;
  h->eps = eps;
  h->nrhs_max = o.max_nrhs;
  h->p2p_unit = o.p2p_unit;
  h->tc_kslice_max = o.tc_kslice;
  h->corr_rules32 = o.corr_rules32 ? 1 : 0;
  h->tc_fp16 = (o.mode == BEM_MODE_FMM_MIXED && o.tc_tf32 == 0) ? 1 : 0;
  h->tc_pipeline = o.tc_pipeline;
  h->p2p_ctas = o.p2p_ctas;
  h->p2p_stage = o.p2p_stage ? 1 : 0;
  h->grad_direct = o.grad_direct ? 1 : 0;
  h->p_min = o.p_min;
  h->p_max = o.p_max;
  for (int l = 0; l <= BEM_MAXLEV; ++l) {
    if (o.p_level[l] < 0 || o.p_level[l] > 60) {
      delete h;
      return bem_fail(BEM_ERR_INVALID_ARG, "p_level entries must be in [0, 60]");
    }
    h->p_level[l] = o.p_level[l];
  }
  h->nt = mesh->n_triangles;
  h->nv = mesh->n_vertices;

  auto fail = [&](int rc) {
    std::string m = g_last_error;
    free_handle(h);
    g_last_error = m;
    return rc;
  };
  int rc;
  if ((rc = bem_alloc(h, &h->d_err, 1)) != BEM_OK) return fail(rc);
  if ((rc = bem_alloc(h, &h->p2p_ctr, h->nrhs_max + 2)) != BEM_OK) return fail(rc);
  if (cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess || h->nsm < 1)
    h->nsm = 1;
  {
    // the far field's stream (see the apply): the greatest priority
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->s_far, cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(bem_fail(BEM_ERR_CUDA, std::string("far-field stream: ") + cudaGetErrorString(e)));
  }
  if (cudaMemsetAsync(h->d_err, 0, sizeof(int), s) != cudaSuccess) return fail(bem_fail(BEM_ERR_CUDA, "memset"));

  // device copy of the mesh
  double* dV = nullptr;
  int32_t* dT = nullptr;
  if (mesh->on_device) {
    dV = (double*)mesh->vertices;
    dT = (int32_t*)mesh->triangles;
  } else {
    if (cudaMallocAsync((void**)&dV, 3 * h->nv * sizeof(double), s) != cudaSuccess ||
        cudaMallocAsync((void**)&dT, 3 * h->nt * sizeof(int32_t), s) != cudaSuccess)
      return fail(bem_fail(BEM_ERR_OOM, "mesh copy"));
    if (cudaMemcpyAsync(dV, mesh->vertices, 3 * h->nv * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(dT, mesh->triangles, 3 * h->nt * sizeof(int32_t), cudaMemcpyHostToDevice, s) != cudaSuccess)
      return fail(bem_fail(BEM_ERR_CUDA, "mesh copy"));
  }
  rc = bem_build_geometry(h, dV, dT, s);
  if (!mesh->on_device) {
    cudaFreeAsync(dV, s);
    cudaFreeAsync(dT, s);
  }
  if (rc != BEM_OK) return fail(rc);
  if ((rc = bem_build_tree(h, o.leaf_level, o.leaf_target, s)) != BEM_OK) return fail(rc);
  if (bem_is_fmm(h) && h->L >= 2)
    if ((rc = bem_build_far_field(h, s)) != BEM_OK) return fail(rc);

  // workspaces
  int64_t nt = h->nt, nr = h->nrhs_max;
  if (bem_is_fp64(h)) {
    double4* d;
    if ((rc = bem_alloc(h, &d, nt * nr)) != BEM_OK) return fail(rc);
    h->dens = d;
  } else {
    float4* d;
    if ((rc = bem_alloc(h, &d, nt * nr)) != BEM_OK) return fail(rc);
    h->dens = d;
  }
  if ((rc = bem_alloc(h, &h->zn, 2 * nt * nr)) != BEM_OK) return fail(rc);
  if ((rc = bem_alloc(h, &h->zfar, 2 * nt * nr)) != BEM_OK) return fail(rc);
  if (h->exp_total > 0) {
    size_t n = (size_t)(2 * h->exp_total * nr);
    if (bem_is_fp64(h)) {
      double *a, *b;
      if ((rc = bem_alloc(h, &a, n)) != BEM_OK || (rc = bem_alloc(h, &b, n)) != BEM_OK) return fail(rc);
      h->Mexp = a;
      h->Lexp = b;
    } else {
      float *a, *b;
      if ((rc = bem_alloc(h, &a, n)) != BEM_OK || (rc = bem_alloc(h, &b, n)) != BEM_OK) return fail(rc);
      h->Mexp = a;
      h->Lexp = b;
    }
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(bem_fail(BEM_ERR_CUDA, "setup synchronise"));
  if ((rc = bem_check_device_error(h, s)) != BEM_OK) return fail(rc);
  *out = h;
  return BEM_OK;
}

static int check_apply_args(bem_handle* h, int nrhs, int dtype, int flags) {
  if (!h) return bem_fail(BEM_ERR_INVALID_ARG, "handle is NULL");
  if (nrhs < 1 || nrhs > h->nrhs_max) return bem_fail(BEM_ERR_INVALID_ARG, "nrhs out of [1, max_nrhs]");
  if (dtype != BEM_C64 && dtype != BEM_C128) return bem_fail(BEM_ERR_INVALID_ARG, "dtype must be BEM_C64 or BEM_C128");
  if (flags & ~(BEM_APPLY_NO_HALF | BEM_HOST_BUFFERS)) return bem_fail(BEM_ERR_INVALID_ARG, "unknown flags");
  return BEM_OK;
}

static int ensure_io(bem_handle* h) {
  if (h->io_x) return BEM_OK;
  size_t n = 2 * (size_t)h->nt * h->nrhs_max;
  double *a, *b, *c;
  BEM_TRY(bem_alloc(h, &a, n));
  BEM_TRY(bem_alloc(h, &b, n));
  BEM_TRY(bem_alloc(h, &c, n));
  h->io_x = a;
  h->io_y = b;
  h->io_z = c;
  return BEM_OK;
}

int bem_apply(bem_handle* h, int nrhs, int dtype, const void* x, const void* y, void* z, int flags, void* stream) {
  g_last_error.clear();
  BEM_TRY(check_apply_args(h, nrhs, dtype, flags));
  if (!z) return bem_fail(BEM_ERR_INVALID_ARG, "z is NULL");
  if ((x && x == z) || (y && y == z)) return bem_fail(BEM_ERR_INVALID_ARG, "z must not alias x or y");
  cudaStream_t s = (cudaStream_t)stream;
  int half = (flags & BEM_APPLY_NO_HALF) ? 0 : 1;
  if (flags & BEM_HOST_BUFFERS) {
    BEM_TRY(ensure_io(h));
    size_t bytes = (size_t)nrhs * h->nt * (dtype == BEM_C128 ? 16 : 8);
    const void* dx = nullptr;
    const void* dy = nullptr;
    if (x) {
      BEM_CUDA(cudaMemcpyAsync(h->io_x, x, bytes, cudaMemcpyHostToDevice, s));
      dx = h->io_x;
    }
    if (y) {
      BEM_CUDA(cudaMemcpyAsync(h->io_y, y, bytes, cudaMemcpyHostToDevice, s));
      dy = h->io_y;
    }
    h->launches_last_apply = 0;
    int pr = bem_prof_begin(h, s);
    BEM_TRY(bem_prologue(h, nrhs, dtype, dx, dy, s));
    bem_prof_end(h, pr, 0, 1, s);
    BEM_TRY(bem_apply_sorted(h, nrhs, s));
    pr = bem_prof_begin(h, s);
    BEM_TRY(bem_epilogue(h, nrhs, dtype, dx, h->io_z, half, s));
    bem_prof_end(h, pr, 8, 1, s);
    BEM_CUDA(cudaMemcpyAsync(z, h->io_z, bytes, cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    return BEM_OK;
  }
  h->launches_last_apply = 0;
  int pr = bem_prof_begin(h, s);
  BEM_TRY(bem_prologue(h, nrhs, dtype, x, y, s));
  bem_prof_end(h, pr, 0, 1, s);
  BEM_TRY(bem_apply_sorted(h, nrhs, s));
  pr = bem_prof_begin(h, s);
  BEM_TRY(bem_epilogue(h, nrhs, dtype, x, z, half, s));
  bem_prof_end(h, pr, 8, 1, s);
  return BEM_OK;
}

int bem_profile(bem_handle* h, int enable) {
  g_last_error.clear();
  if (!h) return bem_fail(BEM_ERR_INVALID_ARG, "handle is NULL");
  BEM_CUDA(cudaDeviceSynchronize());
  for (auto& r : h->prof) {
    h->ev_pool.push_back(r.a);
    h->ev_pool.push_back(r.b);
  }
  h->prof.clear();
  h->prof_on = enable ? 1 : 0;
  return BEM_OK;
}

int bem_profile_read(bem_handle* h, double* ms, int64_t* launches, int nstages) {
  g_last_error.clear();
  if (!h || !ms || nstages < 0) return bem_fail(BEM_ERR_INVALID_ARG, "NULL argument");
  for (int i = 0; i < nstages; ++i) {
    ms[i] = 0.0;
    if (launches) launches[i] = 0;
  }
  for (auto& r : h->prof) {
    if (r.stage < 0 || r.stage >= nstages) continue;
    BEM_CUDA(cudaEventSynchronize(r.b));
    float t = 0.f;
    BEM_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
    ms[r.stage] += t;
    if (launches) launches[r.stage] += r.launches;
  }
  return BEM_OK;
}

int bem_apply_adjoint(bem_handle* h, int nrhs, int dtype, const void* g, void* gx, void* gy, int flags,
                      void* stream) {
  g_last_error.clear();
  BEM_TRY(check_apply_args(h, nrhs, dtype, flags));
  if (flags & BEM_HOST_BUFFERS) return bem_fail(BEM_ERR_INVALID_ARG, "bem_apply_adjoint takes device buffers only");
  if (!g) return bem_fail(BEM_ERR_INVALID_ARG, "g is NULL");
  if (!gx && !gy) return bem_fail(BEM_ERR_INVALID_ARG, "gx and gy are both NULL");
  if (gx == g || gy == g || (gx && gx == gy)) return bem_fail(BEM_ERR_INVALID_ARG, "outputs must not alias");
  cudaStream_t s = (cudaStream_t)stream;
  int half = (flags & BEM_APPLY_NO_HALF) ? 0 : 1;
  return bem_adjoint_sorted(h, nrhs, dtype, g, gx, gy, half, s);
}

int bem_gmres_solve(bem_handle* h, int nrhs, int dtype, const void* b, void* x, double tol, int max_iter, int restart,
                    int flags, int* iters_out, double* relres_out, void* stream) {
  g_last_error.clear();
  BEM_TRY(check_apply_args(h, nrhs, dtype, 0));
  if (!b || !x) return bem_fail(BEM_ERR_INVALID_ARG, "b or x is NULL");
  if (!(tol > 0.0) || max_iter < 1 || restart < 1) return bem_fail(BEM_ERR_INVALID_ARG, "bad tol/max_iter/restart");
  if (flags & ~(BEM_GMRES_USE_X0 | BEM_GMRES_HOST_LOOP | BEM_GMRES_GRAPH_ONLY))
    return bem_fail(BEM_ERR_INVALID_ARG, "flags: BEM_GMRES_USE_X0 | BEM_GMRES_HOST_LOOP | BEM_GMRES_GRAPH_ONLY");
  return bem_gmres(h, nrhs, dtype, b, x, tol, max_iter, restart, flags, iters_out, relres_out, (cudaStream_t)stream);
}

int bem_gmres_solve_coupled(bem_handle* h, int nrhs, int dtype, const void* b, void* x, double tol, int max_iter,
                            int restart, bem_coupling_fn cb, void* cb_ctx, double* cx, double* cy, int flags,
                            int* iters_out, double* relres_out, void* stream) {
  g_last_error.clear();
  BEM_TRY(check_apply_args(h, nrhs, dtype, 0));
  if (!b || !x || !cb || !cx || !cy) return bem_fail(BEM_ERR_INVALID_ARG, "b, x, cb, cx or cy is NULL");
  if (((uintptr_t)cx | (uintptr_t)cy) & 15) return bem_fail(BEM_ERR_INVALID_ARG, "cx and cy must be 16-byte aligned");
  // byte extents: cx, cy complex128; b, x in the caller's dtype
  const uintptr_t nc = (uintptr_t)nrhs * h->nt * 16, nb = (uintptr_t)nrhs * h->nt * (dtype == BEM_C128 ? 16 : 8);
  const uintptr_t lo[4] = {(uintptr_t)cx, (uintptr_t)cy, (uintptr_t)b, (uintptr_t)x}, len[4] = {nc, nc, nb, nb};
  for (int a = 0; a < 2; ++a)
    for (int o = a + 1; o < 4; ++o)
      if (lo[a] < lo[o] + len[o] && lo[o] < lo[a] + len[a])
        return bem_fail(BEM_ERR_INVALID_ARG, "cx or cy overlaps b, x or the other");
  if (!(tol > 0.0) || max_iter < 1 || restart < 1) return bem_fail(BEM_ERR_INVALID_ARG, "bad tol/max_iter/restart");
  if (flags & ~(BEM_GMRES_USE_X0 | BEM_GMRES_HOST_LOOP | BEM_GMRES_GRAPH_ONLY))
    return bem_fail(BEM_ERR_INVALID_ARG, "flags: BEM_GMRES_USE_X0 | BEM_GMRES_HOST_LOOP | BEM_GMRES_GRAPH_ONLY");
  if (flags & BEM_GMRES_GRAPH_ONLY)
    return bem_fail(BEM_ERR_UNSUPPORTED, "a coupled solve runs the host loop: its callback cannot be captured");
  return bem_gmres_coupled(h, nrhs, dtype, b, x, tol, max_iter, restart, cb, cb_ctx, cx, cy, flags, iters_out,
                           relres_out, (cudaStream_t)stream);
}

int bem_info(bem_handle* h, int key, int64_t* value) {
  g_last_error.clear();
  if (!h || !value) return bem_fail(BEM_ERR_INVALID_ARG, "NULL argument");
  int L = h->L;
  switch (key) {
    case BEM_INFO_N: *value = h->nt; return BEM_OK;
    case BEM_INFO_LEAF_LEVEL: *value = L; return BEM_OK;
    case BEM_INFO_N_LEAVES: *value = h->nleaf_all; return BEM_OK;
    case BEM_INFO_P2P_PAIRS: *value = bem_is_fmm(h) ? h->p2p_pairs : h->nt * h->nt; return BEM_OK;
    case BEM_INFO_CORR_NNZ: *value = h->corr_nnz; return BEM_OK;
    case BEM_INFO_M2L_PAIRS: {
      int64_t v = 0;
      for (int l = 2; l <= L; ++l) v += h->m2l[l].npairs;
      *value = v;
      return BEM_OK;
    }
    case BEM_INFO_M2L_FLOPS: {
      int64_t v = 0;
      for (int l = 2; l <= L; ++l) v += h->m2l[l].flops;
      *value = v;
      return BEM_OK;
    }
    case BEM_INFO_P_LEAF: *value = (L >= 2) ? h->lev[L].p : 0; return BEM_OK;
    case BEM_INFO_P_TOP: *value = (L >= 2) ? h->lev[2].p : 0; return BEM_OK;
    case BEM_INFO_MODE: *value = h->mode; return BEM_OK;
    case BEM_INFO_DEVICE_BYTES: *value = (int64_t)h->bytes; return BEM_OK;
    case BEM_INFO_LAUNCHES_LAST_APPLY: *value = h->launches_last_apply; return BEM_OK;
    case BEM_INFO_M2M_FLOPS:
    case BEM_INFO_L2L_FLOPS: {
      int64_t v = 0;
      for (int l = 2; l < L; ++l) v += (key == BEM_INFO_M2M_FLOPS ? h->m2m[l] : h->l2l[l]).flops;
      *value = v;
      return BEM_OK;
    }
    case BEM_INFO_P2M_BYTES: *value = h->row_total * 3 * (bem_is_fp64(h) ? 16 : 8); return BEM_OK;
    case BEM_INFO_ADAPTIVE: *value = h->adaptive; return BEM_OK;
    case BEM_INFO_ROW_COEFFS: *value = h->row_total; return BEM_OK;
    case BEM_INFO_W_PAIRS: *value = h->w_nnz; return BEM_OK;
    case BEM_INFO_X_PAIRS: {
      int64_t v = 0;
      for (int l = 0; l <= L; ++l) v += h->x_n[l];
      *value = v;
      return BEM_OK;
    }
    case BEM_INFO_NEAR_LIST: *value = h->u_nnz; return BEM_OK;
    case BEM_INFO_W_EVALS: *value = h->w_evals; return BEM_OK;
    case BEM_INFO_X_EVALS: *value = h->x_evals; return BEM_OK;
    case BEM_INFO_EXP_TOTAL: *value = h->exp_total; return BEM_OK;
    case BEM_INFO_TC_KIND:
      *value = (!bem_is_fmm(h) || bem_is_fp64(h)) ? 0 : (h->mode == BEM_MODE_FMM_TF32 ? 3 : (h->tc_fp16 ? 1 : 2));
      return BEM_OK;
    default:
      if (key >= BEM_INFO_ORDER_OF_LEVEL && key <= BEM_INFO_ORDER_OF_LEVEL + BEM_MAXLEV) {
        int l = key - BEM_INFO_ORDER_OF_LEVEL;
        *value = (l >= 2 && l <= L && bem_is_fmm(h)) ? h->lev[l].p : 0;
        return BEM_OK;
      }
      if (key >= BEM_INFO_BOXES_OF_LEVEL && key <= BEM_INFO_BOXES_OF_LEVEL + BEM_MAXLEV) {
        int l = key - BEM_INFO_BOXES_OF_LEVEL;
        *value = (l <= L && !h->lev.empty()) ? h->lev[l].nbox : 0;
        return BEM_OK;
      }
      if (key >= BEM_INFO_EXP_BASE_OF_LEVEL && key <= BEM_INFO_EXP_BASE_OF_LEVEL + BEM_MAXLEV) {
        int l = key - BEM_INFO_EXP_BASE_OF_LEVEL;
        *value = (l >= 2 && l <= L && bem_is_fmm(h)) ? h->lev[l].exp_base : 0;
        return BEM_OK;
      }
      if (key >= BEM_INFO_LEAVES_OF_LEVEL && key <= BEM_INFO_LEAVES_OF_LEVEL + BEM_MAXLEV) {
        int l = key - BEM_INFO_LEAVES_OF_LEVEL;
        *value = (l <= L && !h->lev.empty()) ? h->lev[l].nleaf : 0;
        return BEM_OK;
      }
      return bem_fail(BEM_ERR_INVALID_ARG, "unknown info key");
  }
}

}  // extern "C"
