// bem_apply.cu -- the hot path: z = (1/2 I - D) x + S y  (Section 2.3, step 2(c)).
//
// Stages of one apply (all on the caller's stream):
//   prologue  : gather x, y into octree order, weighted by w_j = A_j/(12 pi)
//   P2P       : regular-rule near field, leaf box against its 27 colleagues,
//               FP32 (range-reduced sincos) or FP64
//   correction: CSR SpMV with the FP64-built near-singular / self corrections
//   P2M       : leaf multipoles from the stored per-element rows (HBM stream)
//   M2M, M2L, L2L : one grouped kernel, gather -> dense complex tile GEMM with
//               the translation matrix of the group -> scatter-add
//   L2P       : far field at the centroids from the stored per-element rows
//   epilogue  : z = 1/2 x + near + far, back to the caller's order and dtype
#include <algorithm>

#include "bem_common.cuh"

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename R>
struct V4of;
template <>
struct V4of<float> {
  typedef float4 T;
};
template <>
struct V4of<double> {
  typedef double4 T;
};

// ---------------------------------------------------------------- prologue --
template <typename Rin, typename V4>
__global__ void k_prologue(int64_t nt, int nrhs, const int* __restrict__ perm, const double* __restrict__ wgt,
                           const Rin* __restrict__ x, const Rin* __restrict__ y, V4* dens) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nt) return;
  int64_t o = perm[s];
  double w = wgt[s];
  for (int r = 0; r < nrhs; ++r) {
    int64_t io = 2 * ((int64_t)r * nt + o);
    V4 d;
    d.x = y ? (w * (double)y[io]) : 0.0;
    d.y = y ? (w * (double)y[io + 1]) : 0.0;
    d.z = x ? (w * (double)x[io]) : 0.0;
    d.w = x ? (w * (double)x[io + 1]) : 0.0;
    dens[(int64_t)r * nt + s] = d;
  }
}

// ---------------------------------------------------------------- epilogue --
template <typename Rout, typename Rin>
__global__ void k_epilogue(int64_t nt, int nrhs, const int* __restrict__ perm, const Rin* __restrict__ x, int half,
                           const double* __restrict__ zn, const double* __restrict__ zfar, Rout* z) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nt) return;
  int64_t o = perm[s];
  for (int r = 0; r < nrhs; ++r) {
    int64_t is = 2 * ((int64_t)r * nt + s), io = 2 * ((int64_t)r * nt + o);
    double re = zn[is], im = zn[is + 1];
    if (zfar) {
      re += zfar[is];
      im += zfar[is + 1];
    }
    if (half && x) {
      re += 0.5 * (double)x[io];
      im += 0.5 * (double)x[io + 1];
    }
    z[io] = (Rout)re;
    z[io + 1] = (Rout)im;
  }
}

// ----------------------------------------------------------- kernel pieces --
// exp(i kr) for FP32: Cody-Waite reduction by 2 pi (two-term split) then the
// hardware sin/cos on |t| <= pi.
__device__ __forceinline__ void sincos_2pi_reduced(float kr, float* sn, float* cs) {
  const float inv2pi = 0.15915494309189535f;
  const float c_hi = 6.28125f;                 // 2 pi split: exact leading part
  const float c_lo = 1.9353071795864769e-3f;   // 2 pi - 6.28125
  float q = rintf(kr * inv2pi);
  float t = fmaf(-q, c_hi, kr);
  t = fmaf(-q, c_lo, t);
  __sincosf(t, sn, cs);
}

// accumulate the regular-rule contribution of one source point
template <typename R>
__device__ __forceinline__ void p2p_point(R dx, R dy, R dz, R nx, R ny, R nz, R k, R sre, R sim, R tre, R tim,
                                          R& are, R& aim);

template <>
__device__ __forceinline__ void p2p_point<float>(float dx, float dy, float dz, float nx, float ny, float nz, float k,
                                                 float sre, float sim, float tre, float tim, float& are, float& aim) {
  float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  float rinv = rsqrtf(r2);
  float r = r2 * rinv;
  float kr = k * r;
  float sn, cs;
  sincos_2pi_reduced(kr, &sn, &cs);
  float gre = rinv * cs, gim = rinv * sn;  // exp(ikr)/r
  float dn = fmaf(dx, nx, fmaf(dy, ny, dz * nz));
  float f = dn * rinv * rinv;              // (y-x).n / r^2 ; times g gives the /r^3
  // (ikr - 1) exp(ikr)/r = (-g_re - kr g_im) + i (kr g_re - g_im)
  float hre = fmaf(-kr, gim, -gre), him = fmaf(kr, gre, -gim);
  hre *= f;
  him *= f;
  are = fmaf(gre, sre, are);
  are = fmaf(-gim, sim, are);
  aim = fmaf(gre, sim, aim);
  aim = fmaf(gim, sre, aim);
  are = fmaf(-hre, tre, are);
  are = fmaf(him, tim, are);
  aim = fmaf(-hre, tim, aim);
  aim = fmaf(-him, tre, aim);
}

template <>
__device__ __forceinline__ void p2p_point<double>(double dx, double dy, double dz, double nx, double ny, double nz,
                                                  double k, double sre, double sim, double tre, double tim,
                                                  double& are, double& aim) {
  double r2 = dx * dx + dy * dy + dz * dz;
  double r = sqrt(r2);
  double rinv = 1.0 / r;
  double kr = k * r;
  double sn, cs;
  sincos(kr, &sn, &cs);
  double gre = rinv * cs, gim = rinv * sn;
  double dn = dx * nx + dy * ny + dz * nz;
  double f = dn * rinv * rinv;
  double hre = (-kr * gim - gre) * f, him = (kr * gre - gim) * f;
  are += gre * sre - gim * sim - hre * tre + him * tim;
  aim += gre * sim + gim * sre - hre * tim - him * tre;
}

// ------------------------------------------------------------- P2P (FMM) --
// One CTA per leaf target box; targets x split factor over 128 threads; source
// elements of each colleague box staged in shared memory, shifted into the
// target box's frame (coordinates are stored relative to their leaf centre).
#define P2P_THREADS 128
template <typename R>
__global__ void __launch_bounds__(P2P_THREADS) k_p2p_fmm(int nleaf, int64_t nt, R k, R wleaf,
                                                         const int* __restrict__ near27, const int* __restrict__ bstart,
                                                         const int* __restrict__ bend, const int* __restrict__ coord,
                                                         const typename V4of<R>::T* __restrict__ tgt,
                                                         const typename V4of<R>::T* __restrict__ src,
                                                         const typename V4of<R>::T* __restrict__ dens,
                                                         double* __restrict__ zn) {
  typedef typename V4of<R>::T V4;
  __shared__ V4 s_src[P2P_THREADS][3];
  __shared__ V4 s_den[P2P_THREADS];
  __shared__ R s_red[2][P2P_THREADS];
  int b = blockIdx.x;
  int r = blockIdx.y;
  int tid = threadIdx.x;
  int t0 = bstart[b], t1 = bend[b];
  int bx = coord[3 * b], by = coord[3 * b + 1], bz = coord[3 * b + 2];
  const V4* dr = dens + (int64_t)r * nt;
  for (int c0 = t0; c0 < t1; c0 += P2P_THREADS) {
    int nc = min(P2P_THREADS, t1 - c0);
    int nsplit = P2P_THREADS / nc;
    int ti = tid % nc, split = tid / nc;
    bool active = split < nsplit;
    V4 tg = tgt[c0 + ti];
    R are = 0, aim = 0;
    for (int slot = 0; slot < 27; ++slot) {
      int sb = near27[27 * b + slot];
      if (sb < 0) continue;
      R shx = (R)((coord[3 * sb] - bx) * (double)wleaf);
      R shy = (R)((coord[3 * sb + 1] - by) * (double)wleaf);
      R shz = (R)((coord[3 * sb + 2] - bz) * (double)wleaf);
      int s0 = bstart[sb], s1 = bend[sb];
      for (int e0 = s0; e0 < s1; e0 += P2P_THREADS) {
        int ne = min(P2P_THREADS, s1 - e0);
        __syncthreads();
        if (tid < ne) {
          for (int q = 0; q < 3; ++q) {
            V4 v = src[3 * (int64_t)(e0 + tid) + q];
            v.x += shx;
            v.y += shy;
            v.z += shz;
            s_src[tid][q] = v;
          }
          s_den[tid] = dr[e0 + tid];
        }
        __syncthreads();
        if (active) {
          for (int e = split; e < ne; e += nsplit) {
            V4 q0 = s_src[e][0], q1 = s_src[e][1], q2 = s_src[e][2];
            V4 dd = s_den[e];
            R nx = q0.w, ny = q1.w, nz = q2.w;
            p2p_point<R>(q0.x - tg.x, q0.y - tg.y, q0.z - tg.z, nx, ny, nz, k, dd.x, dd.y, dd.z, dd.w, are, aim);
            p2p_point<R>(q1.x - tg.x, q1.y - tg.y, q1.z - tg.z, nx, ny, nz, k, dd.x, dd.y, dd.z, dd.w, are, aim);
            p2p_point<R>(q2.x - tg.x, q2.y - tg.y, q2.z - tg.z, nx, ny, nz, k, dd.x, dd.y, dd.z, dd.w, are, aim);
          }
        }
      }
    }
    __syncthreads();
    s_red[0][tid] = active ? are : (R)0;
    s_red[1][tid] = active ? aim : (R)0;
    __syncthreads();
    if (tid < nc) {
      double sre = 0.0, sim = 0.0;
      for (int sp = 0; sp < nsplit; ++sp) {
        sre += (double)s_red[0][tid + sp * nc];
        sim += (double)s_red[1][tid + sp * nc];
      }
      int64_t o = 2 * ((int64_t)r * nt + c0 + tid);
      zn[o] = sre;
      zn[o + 1] = sim;
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------- direct sums --
// One target per thread; all sources streamed through shared memory.  FP32
// partial sums are flushed into FP64 accumulators after every tile.
template <typename R>
__global__ void __launch_bounds__(P2P_THREADS) k_p2p_direct(int64_t nt, R k, const typename V4of<R>::T* __restrict__ tgt,
                                                            const typename V4of<R>::T* __restrict__ src,
                                                            const typename V4of<R>::T* __restrict__ dens,
                                                            double* __restrict__ zn) {
  typedef typename V4of<R>::T V4;
  __shared__ V4 s_src[P2P_THREADS][3];
  __shared__ V4 s_den[P2P_THREADS];
  int r = blockIdx.y;
  int64_t i = blockIdx.x * (int64_t)P2P_THREADS + threadIdx.x;
  const V4* dr = dens + (int64_t)r * nt;
  V4 tg;
  if (i < nt) tg = tgt[i];
  else tg = tgt[0];
  double sre = 0.0, sim = 0.0;
  for (int64_t e0 = 0; e0 < nt; e0 += P2P_THREADS) {
    int ne = (int)min((int64_t)P2P_THREADS, nt - e0);
    __syncthreads();
    if (threadIdx.x < ne) {
      for (int q = 0; q < 3; ++q) s_src[threadIdx.x][q] = src[3 * (e0 + threadIdx.x) + q];
      s_den[threadIdx.x] = dr[e0 + threadIdx.x];
    }
    __syncthreads();
    R are = 0, aim = 0;
    for (int e = 0; e < ne; ++e) {
      V4 q0 = s_src[e][0], q1 = s_src[e][1], q2 = s_src[e][2];
      V4 dd = s_den[e];
      R nx = q0.w, ny = q1.w, nz = q2.w;
      p2p_point<R>(q0.x - tg.x, q0.y - tg.y, q0.z - tg.z, nx, ny, nz, k, dd.x, dd.y, dd.z, dd.w, are, aim);
      p2p_point<R>(q1.x - tg.x, q1.y - tg.y, q1.z - tg.z, nx, ny, nz, k, dd.x, dd.y, dd.z, dd.w, are, aim);
      p2p_point<R>(q2.x - tg.x, q2.y - tg.y, q2.z - tg.z, nx, ny, nz, k, dd.x, dd.y, dd.z, dd.w, are, aim);
    }
    sre += (double)are;
    sim += (double)aim;
  }
  if (i < nt) {
    int64_t o = 2 * ((int64_t)r * nt + i);
    zn[o] = sre;
    zn[o + 1] = sim;
  }
}

// ------------------------------------------------------------- correction --
template <typename V4>
__global__ void k_correction(int64_t nt, const int* __restrict__ ptr, const int* __restrict__ col,
                             const V4* __restrict__ val, const V4* __restrict__ dens, double* __restrict__ zn) {
  int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  int r = blockIdx.y;
  if (i >= nt) return;
  const V4* dr = dens + (int64_t)r * nt;
  double are = 0.0, aim = 0.0;
  for (int e = ptr[i] + lane; e < ptr[i + 1]; e += 32) {
    V4 c = val[e];
    V4 d = dr[col[e]];
    // S (c.x, c.y) * sigma (d.x, d.y) - D (c.z, c.w) * tau (d.z, d.w)
    are += (double)c.x * d.x - (double)c.y * d.y - (double)c.z * d.z + (double)c.w * d.w;
    aim += (double)c.x * d.y + (double)c.y * d.x - (double)c.z * d.w - (double)c.w * d.z;
  }
  for (int o = 16; o > 0; o >>= 1) {
    are += __shfl_xor_sync(0xffffffffu, are, o);
    aim += __shfl_xor_sync(0xffffffffu, aim, o);
  }
  if (lane == 0) {
    int64_t o = 2 * ((int64_t)r * nt + i);
    zn[o] += are;
    zn[o + 1] += aim;
  }
}

// -------------------------------------------------------------------- P2M --
template <typename R>
__global__ void k_p2m(int nleaf, int64_t nt, int P, const int* __restrict__ bstart, const int* __restrict__ bend,
                      const R* __restrict__ rows_ab, const typename V4of<R>::T* __restrict__ dens, int64_t exp_base,
                      int64_t exp_stride, R* __restrict__ M) {
  typedef typename V4of<R>::T V4;
  int b = blockIdx.x, r = blockIdx.y;
  const V4* dr = dens + (int64_t)r * nt;
  for (int e = threadIdx.x; e < P; e += blockDim.x) {
    R are = 0, aim = 0;
    for (int j = bstart[b]; j < bend[b]; ++j) {
      const R* ab = rows_ab + 2 * ((int64_t)j * 2 * P);
      R a_re = ab[2 * e], a_im = ab[2 * e + 1];
      R b_re = ab[2 * (P + e)], b_im = ab[2 * (P + e) + 1];
      V4 d = dr[j];
      are += a_re * d.x - a_im * d.y - b_re * d.z + b_im * d.w;
      aim += a_re * d.y + a_im * d.x - b_re * d.w - b_im * d.z;
    }
    R* out = M + 2 * ((int64_t)r * exp_stride + exp_base + (int64_t)b * P + e);
    out[0] = are;
    out[1] = aim;
  }
}

// -------------------------------------------------------------------- L2P --
template <typename R>
__global__ void k_l2p(int64_t nt, int P, const int* __restrict__ leaf_of, const R* __restrict__ rows_r,
                      const R* __restrict__ Lexp, int64_t exp_base, int64_t exp_stride, double* __restrict__ zfar) {
  int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  int r = blockIdx.y;
  if (i >= nt) return;
  int b = leaf_of[i];
  const R* row = rows_r + 2 * (i * P);
  const R* Lb = Lexp + 2 * ((int64_t)r * exp_stride + exp_base + (int64_t)b * P);
  R are = 0, aim = 0;
  for (int e = lane; e < P; e += 32) {
    R x = row[2 * e], y = row[2 * e + 1], lr = Lb[2 * e], li = Lb[2 * e + 1];
    are += x * lr - y * li;
    aim += x * li + y * lr;
  }
  for (int o = 16; o > 0; o >>= 1) {
    are += __shfl_xor_sync(0xffffffffu, are, o);
    aim += __shfl_xor_sync(0xffffffffu, aim, o);
  }
  if (lane == 0) {
    int64_t o = 2 * ((int64_t)r * nt + i);
    zfar[o] = (double)are;
    zfar[o + 1] = (double)aim;
  }
}

// ------------------------------------------------ grouped translation GEMM --
// For every job (group g, pairs [p0, p0+np), rows [row0, row0+64)):
//   dst[dst_off[c] + row] += sum_k T_g[row][k] * src[src_off[c] + k]
// 64x64 complex output tile per CTA, 256 threads with 4x4 complex micro-tiles.
#define GT_M 64
#define GT_N 64
#define GT_K 16
template <typename R>
__global__ void __launch_bounds__(256) k_grouped_gemm(const int4* __restrict__ jobs, const int* __restrict__ grows,
                                                     const int* __restrict__ gcols, const int64_t* __restrict__ gmat,
                                                     const R* __restrict__ mats, const int* __restrict__ src_off,
                                                     const int* __restrict__ dst_off, const R* __restrict__ src,
                                                     R* __restrict__ dst, int64_t exp_stride) {
  __shared__ cpx<R> As[GT_K][GT_M];
  __shared__ cpx<R> Bs[GT_K][GT_N];
  __shared__ int s_src[GT_N], s_dst[GT_N];
  int4 job = jobs[blockIdx.x];
  int r = blockIdx.y;
  int g = job.x, p0 = job.y, np = job.z, row0 = job.w;
  int rows = grows[g], cols = gcols[g];
  const cpx<R>* T = (const cpx<R>*)(mats) + gmat[g];
  const cpx<R>* S = (const cpx<R>*)(src) + (int64_t)r * exp_stride;
  cpx<R>* D = (cpx<R>*)(dst) + (int64_t)r * exp_stride;
  int tid = threadIdx.x;
  if (tid < GT_N) {
    s_src[tid] = tid < np ? src_off[p0 + tid] : -1;
    s_dst[tid] = tid < np ? dst_off[p0 + tid] : -1;
  }
  int ty = tid >> 4, tx = tid & 15;
  cpx<R> acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = cmk((R)0, (R)0);
  __syncthreads();
  int lr = tid >> 2, lk = (tid & 3) * 4;  // loader: row/pair lr, k offset lk..lk+3
  for (int k0 = 0; k0 < cols; k0 += GT_K) {
    // A tile
    {
      int row = row0 + lr;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int kk = k0 + lk + q;
        cpx<R> v = cmk((R)0, (R)0);
        if (row < rows && kk < cols) v = T[(int64_t)row * cols + kk];
        As[lk + q][lr] = v;
      }
      int so = s_src[lr];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int kk = k0 + lk + q;
        cpx<R> v = cmk((R)0, (R)0);
        if (so >= 0 && kk < cols) v = S[so + kk];
        Bs[lk + q][lr] = v;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GT_K; ++kk) {
      cpx<R> a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[kk][ty * 4 + q];
        b[q] = Bs[kk][tx * 4 + q];
      }
#pragma unroll
      for (int ii = 0; ii < 4; ++ii)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          acc[ii][jj].re += a[ii].re * b[jj].re - a[ii].im * b[jj].im;
          acc[ii][jj].im += a[ii].re * b[jj].im + a[ii].im * b[jj].re;
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) {
    int c = tx * 4 + jj;
    int dof = s_dst[c];
    if (dof < 0) continue;
#pragma unroll
    for (int ii = 0; ii < 4; ++ii) {
      int row = row0 + ty * 4 + ii;
      if (row < rows) {
        R* p = (R*)(D + dof + row);
        atomicAdd(p, acc[ii][jj].re);
        atomicAdd(p + 1, acc[ii][jj].im);
      }
    }
  }
}

// ----------------------------------------------------------------- driver --
template <typename R>
static int run_grouped(bem_handle* h, GroupedOp& op, const void* src, void* dst, int nrhs, cudaStream_t s) {
  if (op.njobs == 0) return BEM_OK;
  dim3 grid(op.njobs, nrhs);
  k_grouped_gemm<R><<<grid, 256, 0, s>>>(op.d_jobs, op.d_group_rows, op.d_group_cols, op.d_group_mat,
                                         (const R*)h->mats, op.d_src_off, op.d_dst_off, (const R*)src, (R*)dst,
                                         h->exp_total);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

template <typename R>
static int apply_sorted_impl(bem_handle* h, int nrhs, cudaStream_t s) {
  typedef typename V4of<R>::T V4;
  int64_t nt = h->nt;
  const V4* dens = (const V4*)h->dens;
  const V4* tgt = (const V4*)(sizeof(R) == 4 ? (const void*)h->tgt32 : (const void*)h->tgt64);
  const V4* src = (const V4*)(sizeof(R) == 4 ? (const void*)h->src32 : (const void*)h->src64);
  bool fmm = bem_is_fmm(h);
  int L = h->L;
  // near field
  int pr = bem_prof_begin(h, s);
  if (fmm) {
    LevelInfo& lf = h->lev[L];
    dim3 grid(lf.nbox, nrhs);
    k_p2p_fmm<R><<<grid, P2P_THREADS, 0, s>>>(lf.nbox, nt, (R)h->k, (R)lf.w, h->near27, lf.start, lf.end, lf.coord,
                                              tgt, src, dens, h->zn);
  } else {
    dim3 grid(nblk(nt, P2P_THREADS), nrhs);
    k_p2p_direct<R><<<grid, P2P_THREADS, 0, s>>>(nt, (R)h->k, tgt, src, dens, h->zn);
  }
  BEM_CUDA(cudaGetLastError());
  bem_prof_end(h, pr, 1, 1, s);
  pr = bem_prof_begin(h, s);
  {
    dim3 grid(nblk(nt * 32, 256), nrhs);
    k_correction<V4><<<grid, 256, 0, s>>>(nt, h->corr_ptr, h->corr_col, (const V4*)h->corr_val, dens, h->zn);
    BEM_CUDA(cudaGetLastError());
  }
  bem_prof_end(h, pr, 2, 1, s);
  if (!fmm || L < 2) {
    BEM_CUDA(cudaMemsetAsync(h->zfar, 0, sizeof(double) * 2 * nt * nrhs, s));
    return BEM_OK;
  }
  // far field
  size_t esz = 2 * sizeof(R);
  LevelInfo& lf = h->lev[L];
  pr = bem_prof_begin(h, s);
  BEM_CUDA(cudaMemsetAsync(h->Mexp, 0, esz * h->exp_total * nrhs, s));
  BEM_CUDA(cudaMemsetAsync(h->Lexp, 0, esz * h->exp_total * nrhs, s));
  {
    dim3 grid(lf.nbox, nrhs);
    k_p2m<R><<<grid, 128, 0, s>>>(lf.nbox, nt, lf.P, lf.start, lf.end, (const R*)h->p2m_rows, dens, lf.exp_base,
                                  h->exp_total, (R*)h->Mexp);
    BEM_CUDA(cudaGetLastError());
  }
  bem_prof_end(h, pr, 3, 1, s);
  int nl = 0;
  pr = bem_prof_begin(h, s);
  for (int l = L - 1; l >= 2; --l, ++nl) BEM_TRY(run_grouped<R>(h, h->m2m[l], h->Mexp, h->Mexp, nrhs, s));
  bem_prof_end(h, pr, 4, nl, s);
  nl = 0;
  pr = bem_prof_begin(h, s);
  for (int l = 2; l <= L; ++l, ++nl) BEM_TRY(run_grouped<R>(h, h->m2l[l], h->Mexp, h->Lexp, nrhs, s));
  bem_prof_end(h, pr, 5, nl, s);
  nl = 0;
  pr = bem_prof_begin(h, s);
  for (int l = 2; l < L; ++l, ++nl) BEM_TRY(run_grouped<R>(h, h->l2l[l], h->Lexp, h->Lexp, nrhs, s));
  bem_prof_end(h, pr, 6, nl, s);
  pr = bem_prof_begin(h, s);
  {
    dim3 grid(nblk(nt * 32, 256), nrhs);
    k_l2p<R><<<grid, 256, 0, s>>>(nt, lf.P, h->leaf_of, (const R*)h->l2p_rows, (const R*)h->Lexp, lf.exp_base,
                                  h->exp_total, h->zfar);
    BEM_CUDA(cudaGetLastError());
  }
  bem_prof_end(h, pr, 7, 1, s);
  return BEM_OK;
}

int bem_apply_sorted(bem_handle* h, int nrhs, cudaStream_t s) {
  if (bem_is_fp64(h)) return apply_sorted_impl<double>(h, nrhs, s);
  return apply_sorted_impl<float>(h, nrhs, s);
}

int bem_prologue(bem_handle* h, int nrhs, int dtype, const void* x, const void* y, cudaStream_t s) {
  int64_t nt = h->nt;
  unsigned g = nblk(nt, 256);
  bool f64 = bem_is_fp64(h);
  if (dtype == BEM_C128) {
    if (f64)
      k_prologue<double, double4><<<g, 256, 0, s>>>(nt, nrhs, h->perm, h->wgt, (const double*)x, (const double*)y,
                                                    (double4*)h->dens);
    else
      k_prologue<double, float4><<<g, 256, 0, s>>>(nt, nrhs, h->perm, h->wgt, (const double*)x, (const double*)y,
                                                   (float4*)h->dens);
  } else {
    if (f64)
      k_prologue<float, double4><<<g, 256, 0, s>>>(nt, nrhs, h->perm, h->wgt, (const float*)x, (const float*)y,
                                                   (double4*)h->dens);
    else
      k_prologue<float, float4><<<g, 256, 0, s>>>(nt, nrhs, h->perm, h->wgt, (const float*)x, (const float*)y,
                                                  (float4*)h->dens);
  }
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

int bem_epilogue(bem_handle* h, int nrhs, int dtype, const void* x, void* z, int half, cudaStream_t s) {
  int64_t nt = h->nt;
  unsigned g = nblk(nt, 256);
  if (dtype == BEM_C128)
    k_epilogue<double, double><<<g, 256, 0, s>>>(nt, nrhs, h->perm, (const double*)x, half, h->zn, h->zfar,
                                                 (double*)z);
  else
    k_epilogue<float, float><<<g, 256, 0, s>>>(nt, nrhs, h->perm, (const float*)x, half, h->zn, h->zfar, (float*)z);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}
