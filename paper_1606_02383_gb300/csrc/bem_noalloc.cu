// bem_noalloc.cu -- bem_apply_noalloc: the operator apply with its per-call
// scratch in a fixed, library-owned device array instead of the handle's
// workspaces, so the call makes no allocation of any kind.
//
// Who needs it: programs whose device memory is owned by an allocator or pool
// that has already reserved the whole GPU (a cudaMalloc would fail or fragment
// that pool), and latency-critical loops that must not enter the driver's
// allocation path (cudaMalloc and cudaFree can synchronise the device).
//
// The array below is BEM_NOALLOC_SCRATCH_BYTES long.  Every GPU that loads
// this library holds it until the process exits, and every call shares it.
#include <mutex>

#include "bem_common.cuh"

static __device__ __align__(256) unsigned char g_noalloc_scratch[BEM_NOALLOC_SCRATCH_BYTES];

#define BEM_NOALLOC_MAX_DEVICES 64
static void* g_scratch_addr[BEM_NOALLOC_MAX_DEVICES];
static std::mutex g_scratch_mu;

// Device address of the array on the current device.  In host code the name
// g_noalloc_scratch is only a host-side stand-in, never a device address, so
// it is looked up once per device (with that device current) and cached.
static int scratch_address(void** out) {
  int dev = 0;
  BEM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= BEM_NOALLOC_MAX_DEVICES) return bem_fail(BEM_ERR_UNSUPPORTED, "device index above 63");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return bem_fail(BEM_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return BEM_OK;
}

static inline size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

extern "C" int bem_apply_noalloc(bem_handle* h, int nrhs, int dtype, const void* x, const void* y, void* z,
                                 int flags, void* stream) {
  bem_set_error("");
  if (!h) return bem_fail(BEM_ERR_INVALID_ARG, "handle is NULL");
  if (nrhs < 1 || nrhs > h->nrhs_max) return bem_fail(BEM_ERR_INVALID_ARG, "nrhs out of [1, max_nrhs]");
  if (dtype != BEM_C64 && dtype != BEM_C128) return bem_fail(BEM_ERR_INVALID_ARG, "dtype must be BEM_C64 or BEM_C128");
  if (flags & ~BEM_APPLY_NO_HALF)
    return bem_fail(BEM_ERR_INVALID_ARG, "bem_apply_noalloc takes device buffers only (flags: BEM_APPLY_NO_HALF)");
  if (!z) return bem_fail(BEM_ERR_INVALID_ARG, "z is NULL");
  if ((x && x == z) || (y && y == z)) return bem_fail(BEM_ERR_INVALID_ARG, "z must not alias x or y");

  // carve the per-call scratch: weighted densities, near and far partial sums,
  // multipole and local expansions (same layouts as the handle's workspaces)
  bool f64 = bem_is_fp64(h);
  size_t rsz = f64 ? sizeof(double) : sizeof(float);
  size_t n = (size_t)h->nt * nrhs;
  size_t b_dens = round256(n * 4 * rsz);
  size_t b_z = round256(n * 2 * sizeof(double));
  size_t b_exp = round256((size_t)h->exp_total * nrhs * 2 * rsz);
  size_t need = b_dens + 2 * b_z + 2 * b_exp;
  if (need > (size_t)BEM_NOALLOC_SCRATCH_BYTES)
    return bem_fail(BEM_ERR_INVALID_ARG, "bem_apply_noalloc needs " + std::to_string(need) +
                                             " scratch bytes for this mesh and nrhs; the fixed array holds " +
                                             std::to_string((size_t)BEM_NOALLOC_SCRATCH_BYTES));
  void* base = nullptr;
  BEM_TRY(scratch_address(&base));
  unsigned char* p = (unsigned char*)base;

  cudaStream_t s = (cudaStream_t)stream;
  h->launches_last_apply = 0;
  void* keep_dens = h->dens;
  double* keep_zn = h->zn;
  double* keep_zfar = h->zfar;
  void* keep_M = h->Mexp;
  void* keep_L = h->Lexp;
  h->dens = p;
  h->zn = (double*)(p + b_dens);
  h->zfar = (double*)(p + b_dens + b_z);
  h->Mexp = (h->exp_total > 0) ? (void*)(p + b_dens + 2 * b_z) : nullptr;
  h->Lexp = (h->exp_total > 0) ? (void*)(p + b_dens + 2 * b_z + b_exp) : nullptr;
  // the expansions are zeroed inside the apply on every call; densities and
  // partial sums are fully overwritten before they are read
  int half = (flags & BEM_APPLY_NO_HALF) ? 0 : 1;
  int rc = bem_prologue(h, nrhs, dtype, x, y, s);
  if (rc == BEM_OK) rc = bem_apply_sorted(h, nrhs, s);
  if (rc == BEM_OK) rc = bem_epilogue(h, nrhs, dtype, x, z, half, s);
  h->dens = keep_dens;
  h->zn = keep_zn;
  h->zfar = keep_zfar;
  h->Mexp = keep_M;
  h->Lexp = keep_L;
  return rc;
}
