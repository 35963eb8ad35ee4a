// bem_m2l_tc.cu -- the translation GEMMs (M2M, M2L, L2L) of the mixed mode on
// the 5th-generation tensor cores.
//
// Each group applies one complex translation matrix T (P_out x P_in) to many
// gathered expansions (Section 2.3's FMM, translation step).  The complex
// product is written as a real one with interleaved (re, im) rows and columns,
//     [Re out; Im out] = [[Tr, -Ti], [Ti, Tr]] [Re in; Im in],
// so an expansion stored as interleaved complex64 is already a real column of
// length 2 P_in.  FP32 accuracy comes from the 3xTF32 split
// A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi (hi = x rounded to TF32, lo = x - hi),
// all accumulated in FP32 in tensor memory.
//
// One CTA (256 threads) computes a 128-row x 64-pair output tile over a slice
// of at most 8 stages of 32 real K (longer K is split across CTAs):
//   - the A stage (hi and lo, packed at setup in the K-major, no-swizzle core
//     matrix layout) arrives by one bulk asynchronous copy on an mbarrier;
//   - the B stage is gathered by the threads (source expansion of each pair,
//     with the pair's reflection permutation and signs), split into hi/lo and
//     stored in the same layout, then made visible to the async proxy;
//   - one thread issues 4 k-steps x 3 tcgen05.mma (M=128, N=64, K=8) and
//     commits them to an mbarrier that releases the stage;
//   - two stages, and the next stage's B gather is in flight (in registers)
//     while the current stage multiplies.
// The epilogue reads the accumulator with tcgen05.ld (each warp its 32 lanes)
// and scatters with atomic adds, applying the output reflection.
// Every wait is bounded: on expiry the CTA records BEM_DEVERR_TIMEOUT, stops
// issuing work, waits (bounded) for its own copies and MMAs, frees its tensor
// memory and returns.
#include <algorithm>
#include <vector>

#include "bem_common.cuh"

#define TC_N 64         // pairs per tile (MMA N)
#define TC_M 128        // real rows per tile (MMA M)
#define TC_KS 32        // real K per stage (4 MMA k-steps of 8)
#define TC_ABYTES (2 * TC_M * TC_KS * 4)  // hi + lo A stage
#define TC_BBYTES (TC_N * TC_KS * 4)      // one of hi / lo B stage
#define TC_STAGE_BYTES (TC_ABYTES + 2 * TC_BBYTES)
#define TC_SMEM (2 * TC_STAGE_BYTES)

// ----------------------------------------------------------- PTX helpers --
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait: about 2^21 polls with a short sleep (well under a second)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < (1 << 21); ++it) {
    if (mbar_try(bar, parity)) return true;
    __nanosleep(64);
  }
  return false;
}

// K-major, no-swizzle shared-memory matrix descriptor: core matrices of
// 8 rows x 16 bytes; 128 bytes between core matrices along K, 256 bytes
// between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((256u >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the sm_100 family
  return d;
}

// instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = TC_N
__device__ __forceinline__ uint32_t instr_desc() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// offset (bytes) of element (row, k) in a stage block of `rows` rows x 32 K
__device__ __forceinline__ uint32_t core_off(int row, int kk, int rows) {
  int j = kk >> 3, kg = (kk >> 2) & 1, e = kk & 3;
  return (uint32_t)(j * (rows / 8) * 256 + (row >> 3) * 256 + kg * 128 + (row & 7) * 16 + e * 4);
}

// --------------------------------------------------------- setup packing --
// A_real of group g, packed per (row tile, k stage): [hi block | lo block].
__global__ void k_tc_pack(const float* __restrict__ T, int Po, int Pi, int nks, float* out) {
  int rt = blockIdx.x / nks, ks = blockIdx.x % nks;
  float* blk = out + (int64_t)blockIdx.x * (2 * TC_M * TC_KS);
  for (int idx = threadIdx.x; idx < TC_M * TC_KS; idx += blockDim.x) {
    int row = idx / TC_KS, kk = idx % TC_KS;
    int R = rt * TC_M + row, C = ks * TC_KS + kk;
    int q = R >> 1, k = C >> 1;
    float v = 0.f;
    if (q < Po && k < Pi) {
      float tr = T[2 * ((int64_t)q * Pi + k)], ti = T[2 * ((int64_t)q * Pi + k) + 1];
      int pr = R & 1, pc = C & 1;
      v = (pr == pc) ? tr : (pr == 0 ? -ti : ti);
    }
    float hi = tf32_round(v);
    uint32_t o = core_off(row, kk, TC_M) >> 2;
    blk[o] = hi;
    blk[TC_M * TC_KS + o] = v - hi;
  }
}

// ------------------------------------------------------------------ kernel --
#define TC_THREADS 256
#define TC_KSLICE 8  // K stages per job (longer K is split; outputs are accumulated atomically)

// B element held by thread `tid` in register slot q of a stage: a warp covers
// one 8-pair x 4-k core-matrix row block (rr = lane / 4 pairs, e = lane % 4 k),
// so its 32 shared-memory stores hit 32 different banks.
__device__ __forceinline__ void b_slot(int tid, int q, int* c, int* kk) {
  int lane = tid & 31, G = (tid >> 5) + 8 * q;  // G in [0, 64)
  *c = (G & 7) * 8 + (lane >> 2);
  *kk = (G >> 3) * 4 + (lane & 3);
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_grouped_tc(
    const int4* __restrict__ jobs, const int* __restrict__ grows, const int* __restrict__ gcols,
    const int64_t* __restrict__ tcoff, const float* __restrict__ tcA, const int* __restrict__ src_off,
    const int* __restrict__ dst_off, const unsigned char* __restrict__ pflags, const float* __restrict__ src,
    float* __restrict__ dst, int64_t exp_stride, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_a[2];
  __shared__ __align__(8) uint64_t bar_m[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  __shared__ int s_src[TC_N], s_dst[TC_N], s_flg[TC_N];

  const int4 job = jobs[blockIdx.x];
  const int r = blockIdx.y;
  const int g = job.x, p0 = job.y, np = job.z & 255, rt = job.w;
  const int Po = grows[g], Pi = gcols[g];
  const int nks = (2 * Pi + TC_KS - 1) / TC_KS;
  const int ks0 = (job.z >> 8) * TC_KSLICE, ks1 = min(nks, ks0 + TC_KSLICE);
  const float* Ag = tcA + tcoff[g] + (int64_t)rt * nks * (2 * TC_M * TC_KS);
  const float* S = src + 2 * (int64_t)r * exp_stride;
  float* D = dst + 2 * (int64_t)r * exp_stride;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid < TC_N) {
    bool ok = tid < np;
    s_src[tid] = ok ? src_off[p0 + tid] : -1;
    s_dst[tid] = ok ? dst_off[p0 + tid] : -1;
    s_flg[tid] = ok ? (int)pflags[p0 + tid] : 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(TC_N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    s_abort = 0;
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_a[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_m[i])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = instr_desc();
  int issued_a = 0, committed = 0;  // tracked by thread 0 only

  // gather of one B stage into registers (reflection applied)
  float pre[8];
  auto gather = [&](int ks) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int c, kk;
      b_slot(tid, q, &c, &kk);
      int realk = ks * TC_KS + kk;
      int k = realk >> 1, part = realk & 1;
      float v = 0.f;
      int so = s_src[c];
      if (so >= 0 && k < Pi) {
        bool neg;
        int ki = reflect_index(k, s_flg[c], &neg);
        v = S[2 * ((int64_t)so + ki) + part];
        if (neg) v = -v;
      }
      pre[q] = v;
    }
  };
  gather(ks0);

  for (int ks = ks0; ks < ks1; ++ks) {
    const int it = ks - ks0;
    const int st = it & 1;
    unsigned char* sA = smem + st * TC_STAGE_BYTES;
    unsigned char* sBh = sA + TC_ABYTES;
    unsigned char* sBl = sBh + TC_BBYTES;
    // the MMAs that last read this stage must be done before it is rewritten
    if (tid == 0 && it >= 2 && !mbar_wait(smem_u32(&bar_m[st]), ((it >> 1) - 1) & 1)) s_abort = 1;
    __syncthreads();
    if (s_abort) break;
    if (tid == 0) {
      uint32_t bar = smem_u32(&bar_a[st]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(TC_ABYTES) : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       smem_u32(sA)),
                   "l"(Ag + (int64_t)ks * (2 * TC_M * TC_KS)), "r"(TC_ABYTES), "r"(bar)
                   : "memory");
      ++issued_a;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int c, kk;
      b_slot(tid, q, &c, &kk);
      float v = pre[q], hi = tf32_round(v);
      uint32_t o = core_off(c, kk, TC_N);
      *(float*)(sBh + o) = hi;
      *(float*)(sBl + o) = v - hi;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (ks + 1 < ks1) gather(ks + 1);  // in flight while this stage multiplies
    __syncthreads();
    if (tid == 0) {
      if (!mbar_wait(smem_u32(&bar_a[st]), (it >> 1) & 1)) {
        s_abort = 1;
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t a0 = smem_u32(sA), b0 = smem_u32(sBh), b1 = smem_u32(sBl);
#pragma unroll
        for (int j = 0; j < TC_KS / 8; ++j) {
          uint64_t ah = smem_desc(a0 + j * (TC_M / 8) * 256);
          uint64_t al = smem_desc(a0 + TC_M * TC_KS * 4 + j * (TC_M / 8) * 256);
          uint64_t bh = smem_desc(b0 + j * (TC_N / 8) * 256);
          uint64_t bl = smem_desc(b1 + j * (TC_N / 8) * 256);
          mma_tf32(tmem, ah, bh, idesc, (it > 0 || j > 0) ? 1u : 0u);
          mma_tf32(tmem, ah, bl, idesc, 1u);
          mma_tf32(tmem, al, bh, idesc, 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&bar_m[st]))
                     : "memory");
        ++committed;
      }
    }
  }
  // the last commit covers every MMA this thread issued
  if (tid == 0 && committed > 0) {
    int last = committed - 1;
    if (!mbar_wait(smem_u32(&bar_m[last & 1]), (last >> 1) & 1)) s_abort = 1;
  }
  if (tid == 0 && issued_a > committed) {  // a copy landed without its MMAs: let it finish
    int st = (issued_a - 1) & 1;
    mbar_wait(smem_u32(&bar_a[st]), ((issued_a - 1) >> 1) & 1);
  }
  __syncthreads();
  const bool ok = !s_abort;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 and columns [32 (w / 4), + 32)
    const int rowl = 32 * (warp & 3) + lane;
    const int R = rt * TC_M + rowl;
    const int q = R >> 1, part = R & 1;
    const bool vrow = q < Po;
    for (int c0 = 32 * (warp >> 2); c0 < 32 * (warp >> 2) + 32; c0 += 16) {
      uint32_t v[16];
      uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (vrow) {
#pragma unroll
        for (int cc = 0; cc < 16; ++cc) {
          int c = c0 + cc;
          int dof = s_dst[c];
          if (dof < 0) continue;
          bool neg;
          int qi = reflect_index(q, s_flg[c], &neg);
          float val = __uint_as_float(v[cc]);
          atomicAdd(D + 2 * ((int64_t)dof + qi) + part, neg ? -val : val);
        }
      }
    }
  } else if (tid == 0) {
    atomicOr(err, BEM_DEVERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N));
}

// -------------------------------------------------------------------- host --
int bem_build_tc(bem_handle* h, GroupedOp& op, cudaStream_t s) {
  if (op.ngroups == 0) return BEM_OK;
  std::vector<int64_t> off(op.ngroups);
  int64_t tot = 0;
  for (int g = 0; g < op.ngroups; ++g) {
    int nrt = (2 * op.rows[g] + TC_M - 1) / TC_M, nks = (2 * op.cols[g] + TC_KS - 1) / TC_KS;
    off[g] = tot;
    tot += (int64_t)nrt * nks * 2 * TC_M * TC_KS;
  }
  BEM_TRY(bem_alloc(h, &op.tcA, std::max<int64_t>(tot, 4)));
  for (int g = 0; g < op.ngroups; ++g) {
    int nrt = (2 * op.rows[g] + TC_M - 1) / TC_M, nks = (2 * op.cols[g] + TC_KS - 1) / TC_KS;
    k_tc_pack<<<nrt * nks, 256, 0, s>>>((const float*)h->mats + 2 * op.mat_off[g], op.rows[g], op.cols[g], nks,
                                        op.tcA + off[g]);
    BEM_CUDA(cudaGetLastError());
  }
  std::vector<int4> jobs;
  for (int g = 0; g < op.ngroups; ++g) {
    int np = op.pair_start[g + 1] - op.pair_start[g];
    int nrt = (2 * op.rows[g] + TC_M - 1) / TC_M;
    int nks = (2 * op.cols[g] + TC_KS - 1) / TC_KS;
    for (int p0 = 0; p0 < np; p0 += TC_N)
      for (int rt = 0; rt < nrt; ++rt)
        for (int sl = 0; sl * TC_KSLICE < nks; ++sl)
          jobs.push_back(make_int4(g, op.pair_start[g] + p0, std::min(TC_N, np - p0) | (sl << 8), rt));
  }
  op.n_tc_jobs = (int)jobs.size();
  BEM_TRY(bem_alloc(h, &op.d_tc_jobs, std::max<size_t>(jobs.size(), 1)));
  BEM_TRY(bem_alloc(h, &op.d_tc_off, op.ngroups));
  if (!jobs.empty())
    BEM_CUDA(cudaMemcpyAsync(op.d_tc_jobs, jobs.data(), jobs.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
  BEM_CUDA(cudaMemcpyAsync(op.d_tc_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  BEM_CUDA(cudaStreamSynchronize(s));
  return BEM_OK;
}

int bem_run_grouped_tc(bem_handle* h, GroupedOp& op, const void* src, void* dst, int nrhs, cudaStream_t s,
                       int* launches) {
  if (op.n_tc_jobs == 0) return BEM_OK;
  BEM_CUDA(cudaFuncSetAttribute(k_grouped_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  dim3 grid(op.n_tc_jobs, nrhs);
  k_grouped_tc<<<grid, TC_THREADS, TC_SMEM, s>>>(op.d_tc_jobs, op.d_group_rows, op.d_group_cols, op.d_tc_off, op.tcA,
                                          op.d_src_off, op.d_dst_off, op.d_flags, (const float*)src, (float*)dst,
                                          h->exp_total, h->d_err);
  BEM_CUDA(cudaGetLastError());
  ++*launches;
  return BEM_OK;
}
