// bem_inspect.cu -- read-only views of the octree and of the far field's
// intermediate expansions, so that each FMM stage can be checked on its own
// against direct sums (the translation operators of Section 2.3's FMM).
#include <vector>

#include "bem_common.cuh"

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// stored coefficient -> textbook coefficient: M = M~ s_n, L = L~ / s_n with
// s_n = (k w)^n / (2n+1)!! of the coefficient's level
template <typename R>
__global__ void k_unscale(int64_t exp_total, int nrhs, LevTab lt, const double* __restrict__ kw,
                          const R* __restrict__ Mexp, const R* __restrict__ Lexp, double* M, double* L) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= exp_total * nrhs) return;
  const int64_t e = idx % exp_total;
  int lvl = -1;
  for (int l = 2; l <= BEM_MAXLEV; ++l)
    if (lt.P[l] > 0 && e >= lt.base[l]) lvl = l;
  if (lvl < 0) return;
  const int q = (int)((e - lt.base[lvl]) % lt.P[lvl]);
  int n = (int)sqrt((double)q);
  while ((n + 1) * (n + 1) <= q) ++n;
  while (n * n > q) --n;
  double sn = 1.0;
  for (int i = 1; i <= n; ++i) sn *= kw[lvl] / (2.0 * i + 1.0);
  if (M) {
    M[2 * idx] = (double)Mexp[2 * idx] * sn;
    M[2 * idx + 1] = (double)Mexp[2 * idx + 1] * sn;
  }
  if (L) {
    L[2 * idx] = (double)Lexp[2 * idx] / sn;
    L[2 * idx + 1] = (double)Lexp[2 * idx + 1] / sn;
  }
}

__global__ void k_unsort(int64_t nt, int nrhs, const int* __restrict__ perm, const double* __restrict__ zs,
                         double* z) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nt) return;
  const int64_t o = perm[s];
  for (int r = 0; r < nrhs; ++r) {
    z[2 * ((int64_t)r * nt + o)] = zs[2 * ((int64_t)r * nt + s)];
    z[2 * ((int64_t)r * nt + o) + 1] = zs[2 * ((int64_t)r * nt + s) + 1];
  }
}

extern "C" {

int bem_tree_level(bem_handle* h, int level, int* start, int* end, double* centre, unsigned char* flags) {
  bem_set_error("");
  if (!h) return bem_fail(BEM_ERR_INVALID_ARG, "handle is NULL");
  if (level < 0 || level > h->L) return bem_fail(BEM_ERR_INVALID_ARG, "level outside the tree");
  const LevelInfo& lv = h->lev[level];
  const int nb = lv.nbox;
  if (start) BEM_CUDA(cudaMemcpy(start, lv.start, nb * sizeof(int), cudaMemcpyDeviceToHost));
  if (end) BEM_CUDA(cudaMemcpy(end, lv.end, nb * sizeof(int), cudaMemcpyDeviceToHost));
  if (centre) BEM_CUDA(cudaMemcpy(centre, lv.centre, 3 * nb * sizeof(double), cudaMemcpyDeviceToHost));
  if (flags) {
    std::vector<unsigned char> in(nb), it(nb);
    BEM_CUDA(cudaMemcpy(in.data(), lv.intree, nb, cudaMemcpyDeviceToHost));
    BEM_CUDA(cudaMemcpy(it.data(), lv.internal, nb, cudaMemcpyDeviceToHost));
    for (int b = 0; b < nb; ++b) flags[b] = (unsigned char)((in[b] ? 1 : 0) | (it[b] ? 2 : 0));
  }
  return BEM_OK;
}

int bem_sorted_order(bem_handle* h, int* perm) {
  bem_set_error("");
  if (!h || !perm) return bem_fail(BEM_ERR_INVALID_ARG, "handle or perm is NULL");
  BEM_CUDA(cudaMemcpy(perm, h->perm, h->nt * sizeof(int), cudaMemcpyDeviceToHost));
  return BEM_OK;
}

int bem_far_field(bem_handle* h, int nrhs, int dtype, const void* x, const void* y, double* M, double* L,
                  double* zfar, void* stream) {
  bem_set_error("");
  if (!h) return bem_fail(BEM_ERR_INVALID_ARG, "handle is NULL");
  if (nrhs < 1 || nrhs > h->nrhs_max) return bem_fail(BEM_ERR_INVALID_ARG, "nrhs out of [1, max_nrhs]");
  if (dtype != BEM_C64 && dtype != BEM_C128) return bem_fail(BEM_ERR_INVALID_ARG, "dtype must be BEM_C64 or BEM_C128");
  if (!bem_is_fmm(h) || h->L < 2) return bem_fail(BEM_ERR_UNSUPPORTED, "the handle has no far field");
  cudaStream_t s = (cudaStream_t)stream;
  BEM_TRY(bem_prologue(h, nrhs, dtype, x, y, s));
  BEM_TRY(bem_apply_sorted(h, nrhs, s));
  const LevTab lt = bem_levtab(h);
  double hkw[BEM_MAXLEV + 1];
  for (int l = 0; l <= BEM_MAXLEV; ++l) hkw[l] = (l <= h->L) ? h->k * h->lev[l].w : 1.0;
  double* dkw;
  BEM_CUDA(cudaMallocAsync((void**)&dkw, sizeof(hkw), s));
  BEM_CUDA(cudaMemcpyAsync(dkw, hkw, sizeof(hkw), cudaMemcpyHostToDevice, s));
  if (M || L) {
    const int64_t n = h->exp_total * nrhs;
    if (bem_is_fp64(h))
      k_unscale<double><<<nblk(n, 256), 256, 0, s>>>(h->exp_total, nrhs, lt, dkw, (const double*)h->Mexp,
                                                     (const double*)h->Lexp, M, L);
    else
      k_unscale<float><<<nblk(n, 256), 256, 0, s>>>(h->exp_total, nrhs, lt, dkw, (const float*)h->Mexp,
                                                    (const float*)h->Lexp, M, L);
    BEM_CUDA(cudaGetLastError());
  }
  if (zfar) {
    k_unsort<<<nblk(h->nt, 256), 256, 0, s>>>(h->nt, nrhs, h->perm, h->zfar, zfar);
    BEM_CUDA(cudaGetLastError());
  }
  BEM_CUDA(cudaFreeAsync(dkw, s));
  return bem_check_device_error(h, s);
}

}  // extern "C"
