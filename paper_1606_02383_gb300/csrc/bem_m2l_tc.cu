// bem_m2l_tc.cu -- the translation GEMMs (M2M, M2L, L2L) of the mixed mode on
// the 5th-generation tensor cores.
//
// Each group applies one complex translation matrix T (P_out x P_in) to many
// gathered expansions (Section 2.3's FMM, translation step).  The complex
// product is written as a real one with interleaved (re, im) rows and columns,
//     [Re out; Im out] = [[Tr, -Ti], [Ti, Tr]] [Re in; Im in],
// so an expansion stored as interleaved complex64 is already a real vector of
// length 2 P_in.  FP32 accuracy comes from the 3xTF32 split
// A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi (hi = x rounded to TF32, lo = x - hi),
// all accumulated in FP32 in tensor memory.
//
// The MMA is D[pairs x rows] += E[pairs x K] . T_real[rows x K]^T: M = 128
// pairs of one group, N = up to 256 real output rows, K in stages of 16:
//   - the T stage (hi and lo, packed at setup in the K-major, no-swizzle core
//     matrix layout) arrives by one bulk asynchronous copy on an mbarrier;
//   - the E stage is gathered by the threads (source expansion of every pair,
//     with the pair's reflection permutation and signs), split into hi/lo and
//     stored in the same layout, then made visible to the async proxy; the
//     next stage's gather is in flight in registers while this one multiplies;
//   - one thread issues 2 k-steps x 3 tcgen05.mma (M=128, N<=256, K=8) and
//     commits them to an mbarrier that releases the stage (two stages);
//   - long K is split across CTAs (outputs are accumulated atomically).
// FP16 split (the default of the mixed mode): the same product with
// kind::f16 MMAs (K = 16 per instruction, 32 per stage) on a two-term FP16
// split, A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi.  FP16 keeps 11 significant
// bits like TF32 but only a 5-bit exponent, so every source row (pair) and
// every matrix row is scaled by a power of two that puts its largest entry
// in [2^13, 2^14) before the split; the epilogue multiplies the scales back
// out (exact).  A stage then holds 32 K in the bytes TF32 needs for 16, so the
// matrices stream half the bytes and the pipeline runs half the stages.
// In the epilogue every thread owns one pair (its TMEM lane) and adds that
// pair's outputs to the destination expansion with (re, im) vector atomics,
// applying the output reflection.  Every wait is bounded (about one second of
// SM clocks): on expiry the CTA records BEM_DEVERR_TIMEOUT, stops issuing work,
// waits (bounded) for its own copies and MMAs, frees its tensor memory and
// returns.
#include <algorithm>
#include <vector>

#include <cuda_fp16.h>

#include "bem_common.cuh"

#define TC_M 128        // pairs per tile (MMA M)
#define TC_NMAX 256     // real output rows per tile (MMA N, multiple of 16)
#define TC_KS 16        // real K per stage (2 MMA k-steps of 8)
#define TC_KSLICE 16    // stages per job, at most
#define TC_THREADS 256
#define TC_EBYTES (TC_M * TC_KS * 4)                     // one of hi / lo gathered stage
#define TC_TBYTES_MAX (TC_NMAX * TC_KS * 4)             // one of hi / lo matrix stage
#define TC_STAGE_BYTES (2 * TC_EBYTES + 2 * TC_TBYTES_MAX)
#define TC_SMEM (2 * TC_STAGE_BYTES)

// ----------------------------------------------------------- PTX helpers --
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

// try_wait suspends the thread in hardware until the phase completes or a
// system-defined time window passes, so polling it costs no issue slots
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait: gives up after `limit` SM clocks (default 2^31, about one second)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit = (1LL << 31)) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    if (mbar_try(bar, parity)) return true;
    if (clock64() - t0 > limit) return false;
  }
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

// instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t instr_desc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

// instruction descriptor: D = F32, A = B = F16, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t instr_desc_f16(int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// offset (bytes) of element (row, k) in a stage block of `rows` rows x TC_KS K
__device__ __forceinline__ uint32_t core_off(int row, int kk, int rows) {
  int j = kk >> 3, kg = (kk >> 2) & 1, e = kk & 3;
  return (uint32_t)(j * (rows / 8) * 256 + (row >> 3) * 256 + kg * 128 + (row & 7) * 16 + e * 4);
}
// the same layout by byte position within a row's 64-byte stage (32 FP16 or 16 TF32)
__device__ __forceinline__ uint32_t core_off_b(int row, int byte, int rows) {
  int j = byte >> 5, kg = (byte >> 4) & 1, e = byte & 15;
  return (uint32_t)(j * (rows / 8) * 256 + (row >> 3) * 256 + kg * 128 + (row & 7) * 16 + e);
}

// power of two that puts x's magnitude in [2^13, 2^14) (1 for 0), and its inverse
__host__ __device__ __forceinline__ void f16_scale(float x, float* scale, float* inv) {
  if (!(x > 0.f) || !isfinite(x)) {
    *scale = *inv = 1.f;
    return;
  }
  int ex;
  frexpf(x, &ex);  // x = m 2^ex, m in [0.5, 1)
  *scale = ldexpf(1.f, 14 - ex);
  *inv = ldexpf(1.f, ex - 14);
}

// --------------------------------------------------------- setup packing --
// Rows of n-tile nt: real output rows [256 nt, 256 nt + N) with N the tile's
// width rounded up to 16; per k stage a block [hi N x 16 | lo N x 16].
__host__ __device__ __forceinline__ int tc_ntile_width(int rows_real, int nt) {
  int w = min(TC_NMAX, rows_real - nt * TC_NMAX);
  return (w + 15) & ~15;
}

__global__ void k_tc_pack(const float* __restrict__ T, int Po, int Pi, int nks, int nnt, float* out) {
  int nt = blockIdx.x / nks, ks = blockIdx.x % nks;
  int N = tc_ntile_width(2 * Po, nt);
  float* blk = out + (int64_t)nt * nks * (2 * TC_NMAX * TC_KS) + (int64_t)ks * (2 * N * TC_KS);
  for (int idx = threadIdx.x; idx < N * TC_KS; idx += blockDim.x) {
    int row = idx / TC_KS, kk = idx % TC_KS;
    int R = nt * TC_NMAX + row, C = ks * TC_KS + kk;
    int q = R >> 1, k = C >> 1;
    float v = 0.f;
    if (q < Po && k < Pi) {
      float tr = T[2 * ((int64_t)q * Pi + k)], ti = T[2 * ((int64_t)q * Pi + k) + 1];
      int pr = R & 1, pc = C & 1;
      v = (pr == pc) ? tr : (pr == 0 ? -ti : ti);
    }
    float hi = tf32_round(v);
    uint32_t o = core_off(row, kk, N) >> 2;
    blk[o] = hi;
    blk[N * TC_KS + o] = v - hi;
  }
  (void)nnt;
}

// FP16 packing: rows scaled by rsc[R] (largest entry in [2^13, 2^14)); per
// k stage of 32 a block [hi N x 32 | lo N x 32] halves, in the byte layout of
// the TF32 blocks (64 bytes per row and half).
__global__ void k_tc_rowscale(const float* __restrict__ T, int Po, int Pi, float* rsc, float* rinv) {
  // one warp per output coefficient q (real rows 2q, 2q+1 share the entries)
  const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (q >= Po) return;
  float m = 0.f;
  for (int k = lane; k < Pi; k += 32)
    m = fmaxf(m, fmaxf(fabsf(T[2 * ((int64_t)q * Pi + k)]), fabsf(T[2 * ((int64_t)q * Pi + k) + 1])));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) {
    float sc, iv;
    f16_scale(m, &sc, &iv);
    rsc[2 * q] = rsc[2 * q + 1] = sc;
    rinv[2 * q] = rinv[2 * q + 1] = iv;
  }
}

__global__ void k_tc_pack16(const float* __restrict__ T, int Po, int Pi, int nks, const float* __restrict__ rsc,
                            float* out) {
  int nt = blockIdx.x / nks, ks = blockIdx.x % nks;
  int N = tc_ntile_width(2 * Po, nt);
  unsigned char* blk = (unsigned char*)(out + (int64_t)nt * nks * (2 * TC_NMAX * TC_KS) + (int64_t)ks * (2 * N * TC_KS));
  for (int idx = threadIdx.x; idx < N * 32; idx += blockDim.x) {
    int row = idx / 32, kk = idx % 32;
    int R = nt * TC_NMAX + row, C = ks * 32 + kk;
    int q = R >> 1, k = C >> 1;
    float v = 0.f;
    if (q < Po && k < Pi) {
      float tr = T[2 * ((int64_t)q * Pi + k)], ti = T[2 * ((int64_t)q * Pi + k) + 1];
      int pr = R & 1, pc = C & 1;
      v = ((pr == pc) ? tr : (pr == 0 ? -ti : ti)) * rsc[R];
    }
    const __half hi = __float2half_rn(v);
    const __half lo = __float2half_rn(v - __half2float(hi));
    const uint32_t o = core_off_b(row, 2 * kk, N);
    *(__half*)(blk + o) = hi;
    *(__half*)(blk + N * 64 + o) = lo;
  }
}

// Epilogue of one tile: TMEM lanes hold the tile's 128 pairs, columns its N
// real output rows.  In chunks of 64 columns (32 output coefficients):
//   1. warp w copies lanes 32 (w % 4) .. + 31, columns 32 (w / 4) .. + 31 of
//      the chunk from tensor memory into a shared tile [pair][column] (rows
//      padded to 68 floats: the 16-byte stores of 8 consecutive pairs cover
//      all banks);
//   2. warp w takes pairs w, w + 8, ...: lane j adds coefficient j of the
//      chunk, scaled back (FP16 split), reflected and signed as the pair's
//      flags say, to the pair's destination expansion, so that one warp's
//      atomics fall on one expansion's consecutive coefficients (a few
//      32-byte sectors per instruction instead of one sector per lane).
// `buf` is the kernel's stage memory, free once every copy and MMA is done.
#define TC_EPI_STRIDE 68
template <bool F16>
__device__ __forceinline__ void tc_epilogue(uint32_t tmem, int warp, int lane, unsigned char* buf, const int* s_src,
                                            const int* s_dst, const int* s_flg, const float* __restrict__ escale,
                                            const float* __restrict__ tscale, const int* __restrict__ tsoff, int g,
                                            int Po, int N, int nt, float* __restrict__ D) {
  float* tile = (float*)buf;
  const float* tsg = F16 ? tscale + tsoff[g] : nullptr;
  const int pr = 32 * (warp & 3) + lane;
  for (int c0 = 0; c0 < N; c0 += 64) {
    const int ncol = min(64, N - c0);  // a multiple of 16
    const int cw = 32 * (warp >> 2);   // this warp's columns within the chunk
#pragma unroll
    for (int j = 0; j < 32; j += 8) {
      if (cw + j < ncol) {
        uint32_t v[8];
        const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(c0 + cw + j);
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                     : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float* t = tile + pr * TC_EPI_STRIDE + cw + j;
        *(float4*)t = make_float4(__uint_as_float(v[0]), __uint_as_float(v[1]), __uint_as_float(v[2]),
                                  __uint_as_float(v[3]));
        *(float4*)(t + 4) = make_float4(__uint_as_float(v[4]), __uint_as_float(v[5]), __uint_as_float(v[6]),
                                        __uint_as_float(v[7]));
      }
    }
    __syncthreads();
    // output coefficient of lane j: q = (nt TC_NMAX + c0) / 2 + j = n^2 + n + m
    const int q = (nt * TC_NMAX + c0) / 2 + lane;
    const bool live = 2 * lane < ncol && q < Po;
    int n = (int)sqrtf((float)q);
    if ((n + 1) * (n + 1) <= q) ++n;
    if (n * n > q) --n;
    const int m = q - n * n - n;
    const float ts = (F16 && live) ? tsg[2 * q] : 1.f;
    for (int pc = warp; pc < TC_M; pc += 8) {
      const int dof = s_dst[pc];
      if (dof < 0) continue;
      if (live) {
        const int fl = s_flg[pc];
        const bool neg = ((fl & 1) && (m & 1)) != ((fl & 4) && ((n + m) & 1));
        const bool mflip = ((fl & 1) != 0) != ((fl & 2) != 0);
        float sc = neg ? -1.f : 1.f;
        if (F16) sc *= escale[s_src[pc]] * ts;
        const float2 v = *(const float2*)(tile + pc * TC_EPI_STRIDE + 2 * lane);
        atomicAdd((float2*)(D + 2 * ((int64_t)dof + (mflip ? n * n + n - m : q))), make_float2(sc * v.x, sc * v.y));
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ kernel --
// F16: the FP16-split form (32 K per stage, scaled rows: escale per prepared
// source row, tscale per matrix row at tsoff[g]); otherwise TF32 (16 K per
// stage, nprod = 3 for 3xTF32 or 1 for plain TF32).
template <bool F16>
__global__ void __launch_bounds__(TC_THREADS, 1) k_grouped_tc(
    const int4* __restrict__ jobs, const int* __restrict__ grows, const int* __restrict__ gcols,
    const int64_t* __restrict__ tcoff, const float* __restrict__ tcB, const int* __restrict__ prep_row,
    const int* __restrict__ dst_off, const unsigned char* __restrict__ pflags, const float* __restrict__ prep,
    int row_floats, int nchunk, int rows_per_rhs, float* __restrict__ dst, int64_t exp_stride, int nprod, int kslice,
    int* err, long long wait_limit, int hold_first_copy, const float* __restrict__ escale,
    const float* __restrict__ tscale, const int* __restrict__ tsoff) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_t[2];
  __shared__ __align__(8) uint64_t bar_m[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  __shared__ int s_src[TC_M], s_dst[TC_M], s_flg[TC_M];

  // blocks walk (job, rhs) with the rhs fastest, so the CTAs that read one
  // matrix stage run together and share it through L2
  const int4 job = jobs[blockIdx.x / nchunk];
  const int r = blockIdx.x % nchunk;
  const int g = job.x, p0 = job.y, np = job.z & 255, nt = job.w;
  const int Po = grows[g], Pi = gcols[g];
  const int N = tc_ntile_width(2 * Po, nt);
  constexpr int KSTG = F16 ? 32 : TC_KS;  // K per stage
  const int nks = (2 * Pi + KSTG - 1) / KSTG;
  const int ks0 = (job.z >> 8) * kslice, ks1 = min(nks, ks0 + kslice);
  const float* Tg = tcB + tcoff[g] + (int64_t)nt * nks * (2 * TC_NMAX * TC_KS);
  const uint32_t tbytes = (uint32_t)(2 * N * TC_KS * 4);
  float* D = dst + 2 * (int64_t)r * exp_stride;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid < TC_M) {
    bool ok = tid < np;
    s_src[tid] = ok ? prep_row[p0 + tid] + r * rows_per_rhs : -1;
    s_dst[tid] = ok ? dst_off[p0 + tid] : -1;
    s_flg[tid] = ok ? (int)pflags[p0 + tid] : 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(TC_NMAX));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    s_abort = 0;
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_t[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_m[i])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = F16 ? instr_desc_f16(N) : instr_desc(N);
  int issued_t = 0, committed = 0;  // tracked by thread 0 only

  // gather of one E stage from the prepared rows (reflection and hi/lo split
  // already applied; per stage a pair's row holds [hi 16 | lo 16]).  Item
  // bits: pair (3 low bits), quad (2), pair group (4), half hi/lo (1): a warp
  // covers 8 pairs x 4 quads of one half, i.e. 8 requests of 64 contiguous
  // bytes, and its 16-byte shared stores fill 4 whole 128-byte lines
  auto gather = [&](float4(&pre)[4], int ks) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int item = tid + TC_THREADS * q;  // 0..1023
      const int c = ((item >> 5) & 15) * 8 + (item & 7), quad = (item >> 3) & 3, part = item >> 9;
      const int row = s_src[c];
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (row >= 0) v = *(const float4*)(prep + (int64_t)row * row_floats + ks * (2 * TC_KS) + part * TC_KS + quad * 4);
      pre[q] = v;
    }
  };
  // one bulk copy of matrix stage `it` into buffer it & 1 (thread 0)
  auto issue_t = [&](int it) {
    const uint32_t bar = smem_u32(&bar_t[it & 1]);
    unsigned char* sT = smem + (it & 1) * TC_STAGE_BYTES + 2 * TC_EBYTES;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tbytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(sT)),
                 "l"(Tg + (int64_t)(ks0 + it) * (2 * N * TC_KS)), "r"(tbytes), "r"(bar)
                 : "memory");
    ++issued_t;
  };
  __syncthreads();  // s_src visible
  // Pipeline (two smem buffers, stage it in buffer it & 1): the gather runs two
  // stages ahead in registers (sets pA / pB alternate), and the matrix copy of
  // stage it + 1 is issued as soon as MMA(it - 1) has released its buffer, so
  // a copy has a whole stage of MMA work to land behind.
  const int nstage = ks1 - ks0;
  float4 pA[4], pB[4];
  gather(pA, ks0);
  if (nstage > 1) gather(pB, ks0 + 1);
  // hold_first_copy (diagnostic of the timeout path): stage 0's matrix copy is
  // never issued, so the first matrix-stage wait expires with nothing in flight
  if (tid == 0 && !hold_first_copy) issue_t(0);
  auto body = [&](float4(&cur)[4], int it) -> bool {
    const int st = it & 1;
    unsigned char* sEh = smem + st * TC_STAGE_BYTES;
    unsigned char* sEl = sEh + TC_EBYTES;
    unsigned char* sT = sEl + TC_EBYTES;  // [hi N x 16 | lo N x 16]
    __syncthreads();  // buffer st is free: thread 0 saw MMA(it - 2) complete
    if (s_abort) return false;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int item = tid + TC_THREADS * q;
      const int c = ((item >> 5) & 15) * 8 + (item & 7), quad = (item >> 3) & 3, part = item >> 9;
      *(float4*)((part ? sEl : sEh) + core_off(c, quad * 4, TC_M)) = cur[q];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (it + 2 < nstage) gather(cur, ks0 + it + 2);
    __syncthreads();
    if (tid == 0) {
      if (!mbar_wait(smem_u32(&bar_t[st]), (it >> 1) & 1, wait_limit)) {
        s_abort = 1;
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t e0 = smem_u32(sEh), e1 = smem_u32(sEl), t0 = smem_u32(sT);
#pragma unroll
        for (int j = 0; j < TC_KS / 8; ++j) {
          uint64_t ah = smem_desc(e0 + j * (TC_M / 8) * 256);
          uint64_t al = smem_desc(e1 + j * (TC_M / 8) * 256);
          uint64_t bh = smem_desc(t0 + j * (N / 8) * 256);
          uint64_t bl = smem_desc(t0 + N * TC_KS * 4 + j * (N / 8) * 256);
          if constexpr (F16) {
            mma_f16(tmem, ah, bh, idesc, (it > 0 || j > 0) ? 1u : 0u);
            mma_f16(tmem, ah, bl, idesc, 1u);
            mma_f16(tmem, al, bh, idesc, 1u);
          } else {
            mma_tf32(tmem, ah, bh, idesc, (it > 0 || j > 0) ? 1u : 0u);
            if (nprod == 3) {
              mma_tf32(tmem, ah, bl, idesc, 1u);
              mma_tf32(tmem, al, bh, idesc, 1u);
            }
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&bar_m[st]))
                     : "memory");
        ++committed;
        if (it + 1 < nstage) {
          // buffer st ^ 1 held stage it - 1: wait for its MMAs, then refill it
          if (it >= 1 && !mbar_wait(smem_u32(&bar_m[st ^ 1]), ((it - 1) >> 1) & 1))
            s_abort = 1;
          else
            issue_t(it + 1);
        }
      }
    }
    return true;
  };
  for (int it = 0; it < nstage; it += 2) {
    if (!body(pA, it)) break;
    if (it + 1 < nstage && !body(pB, it + 1)) break;
  }
  if (tid == 0 && committed > 0) {
    int last = committed - 1;
    if (!mbar_wait(smem_u32(&bar_m[last & 1]), (last >> 1) & 1)) s_abort = 1;
  }
  if (tid == 0 && issued_t > committed) {
    int st = (issued_t - 1) & 1;
    mbar_wait(smem_u32(&bar_t[st]), ((issued_t - 1) >> 1) & 1);
  }
  __syncthreads();
  const bool ok = !s_abort;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    tc_epilogue<F16>(tmem, warp, lane, smem, s_src, s_dst, s_flg, escale, tscale, tsoff, g, Po, N, nt, D);
  } else if (tid == 0) {
    atomicOr(err, BEM_DEVERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_NMAX));
}

// ------------------------------------------------- warp-specialised kernel --
// The same tile (job, rhs) and the same MMAs as k_grouped_tc, with the stage
// loop run by three roles on NS shared-memory stages and mbarriers alone:
//   warps 0-3  gather producers: every thread copies 8 of the stage's 1,024
//              16-byte pieces of prepared rows into the core-matrix layout with
//              cp.async (zero-filled for padding pairs); after issuing stage
//              it it waits for its copies of stage it - LAG, fences them to
//              the async proxy and arrives on that stage's gather barrier;
//   warp 4     one thread issues the matrix stage's bulk copy on the matrix
//              barrier (expected bytes);
//   warp 5     one thread waits for both barriers of a stage, issues its MMAs
//              and commits them to the stage's release barrier, which the
//              producers wait on before they refill the stage (NS stages
//              ahead).
// All eight warps then run the epilogue.  Every wait is bounded; on expiry
// the role records the abort, stops issuing, and the CTA drains its own
// copies and MMAs before it frees tensor memory.
#define TC_WS_THREADS 256
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

template <bool F16, int NS, int LAG>
__global__ void __launch_bounds__(TC_WS_THREADS, 1) k_grouped_tc_ws(
    const int4* __restrict__ jobs, const int* __restrict__ grows, const int* __restrict__ gcols,
    const int64_t* __restrict__ tcoff, const float* __restrict__ tcB, const int* __restrict__ prep_row,
    const int* __restrict__ dst_off, const unsigned char* __restrict__ pflags, const float* __restrict__ prep,
    int row_floats, int nchunk, int rows_per_rhs, float* __restrict__ dst, int64_t exp_stride, int nprod, int kslice,
    int* err, long long wait_limit, int hold_first_copy, const float* __restrict__ escale,
    const float* __restrict__ tscale, const int* __restrict__ tsoff) {
  static_assert(LAG >= 1 && LAG < NS, "the gather lag must leave the MMAs a stage of slack");
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_e[NS], bar_t[NS], bar_r[NS];
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_abort;
  __shared__ int s_src[TC_M], s_dst[TC_M], s_flg[TC_M];

  const int4 job = jobs[blockIdx.x / nchunk];
  const int r = blockIdx.x % nchunk;
  const int g = job.x, p0 = job.y, np = job.z & 255, nt = job.w;
  const int Po = grows[g], Pi = gcols[g];
  const int N = tc_ntile_width(2 * Po, nt);
  constexpr int KSTG = F16 ? 32 : TC_KS;
  const int nks = (2 * Pi + KSTG - 1) / KSTG;
  const int ks0 = (job.z >> 8) * kslice, ks1 = min(nks, ks0 + kslice);
  const int nstage = ks1 - ks0;
  const float* Tg = tcB + tcoff[g] + (int64_t)nt * nks * (2 * TC_NMAX * TC_KS);
  const uint32_t tbytes = (uint32_t)(2 * N * TC_KS * 4);
  float* D = dst + 2 * (int64_t)r * exp_stride;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid < TC_M) {
    const bool ok = tid < np;
    s_src[tid] = ok ? prep_row[p0 + tid] + r * rows_per_rhs : -1;
    s_dst[tid] = ok ? dst_off[p0 + tid] : -1;
    s_flg[tid] = ok ? (int)pflags[p0 + tid] : 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(TC_NMAX));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    s_abort = 0;
    for (int i = 0; i < NS; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_e[i])), "r"(TC_M));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_t[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_r[i])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  if (warp < 4) {
    // ---- gather producers: thread t copies items t + 128 q, q = 0..7 ----
    int issued = 0;
    for (int it = 0; it < nstage; ++it) {
      if (s_abort) break;
      const int st = it % NS;
      if (it >= NS && !mbar_wait(smem_u32(&bar_r[st]), ((it / NS) - 1) & 1, wait_limit)) {
        s_abort = 1;
        break;
      }
      unsigned char* sEh = smem + st * TC_STAGE_BYTES;
      unsigned char* sEl = sEh + TC_EBYTES;
      const int ks = ks0 + it;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int item = tid + TC_M * q;  // 0..1023
        const int c = ((item >> 5) & 15) * 8 + (item & 7), quad = (item >> 3) & 3, part = item >> 9;
        const int row = s_src[c];
        const float* src = row >= 0
                               ? prep + (int64_t)row * row_floats + ks * (2 * TC_KS) + part * TC_KS + quad * 4
                               : prep;
        const uint32_t dsm = smem_u32((part ? sEl : sEh) + core_off(c, quad * 4, TC_M));
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dsm), "l"(src), "r"(row >= 0 ? 16 : 0)
                     : "memory");
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      ++issued;
      if (it >= LAG) {
        asm volatile("cp.async.wait_group %0;" ::"n"(LAG) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(smem_u32(&bar_e[(it - LAG) % NS]));
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int j = max(0, issued - LAG); j < issued; ++j) mbar_arrive(smem_u32(&bar_e[j % NS]));
  } else if (warp == 4 && lane == 0) {
    // ---- matrix producer ----
    int last = -1;  // last stage whose copy was issued
    for (int it = 0; it < nstage; ++it) {
      if (s_abort) break;
      const int st = it % NS;
      if (it >= NS && !mbar_wait(smem_u32(&bar_r[st]), ((it / NS) - 1) & 1, wait_limit)) {
        s_abort = 1;
        break;
      }
      // hold_first_copy (diagnostic of the timeout path): stage 0 is never issued
      if (it == 0 && hold_first_copy) continue;
      const uint32_t bar = smem_u32(&bar_t[st]);
      unsigned char* sT = smem + st * TC_STAGE_BYTES + 2 * TC_EBYTES;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tbytes) : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       smem_u32(sT)),
                   "l"(Tg + (int64_t)(ks0 + it) * (2 * N * TC_KS)), "r"(tbytes), "r"(bar)
                   : "memory");
      last = it;
    }
    // the copies still in flight (at most the last NS issued) must land before the CTA ends
    for (int j = max(0, last - NS + 1); j <= last; ++j) {
      if (j == 0 && hold_first_copy) continue;
      if (!mbar_wait(smem_u32(&bar_t[j % NS]), (j / NS) & 1, wait_limit)) s_abort = 1;
    }
  } else if (warp == 5 && lane == 0) {
    // ---- MMA issuer ----
    const uint32_t idesc = F16 ? instr_desc_f16(N) : instr_desc(N);
    int committed = 0;
    for (int it = 0; it < nstage; ++it) {
      if (s_abort) break;
      const int st = it % NS;
      const uint32_t ph = (it / NS) & 1;
      if (!mbar_wait(smem_u32(&bar_t[st]), ph, wait_limit) || !mbar_wait(smem_u32(&bar_e[st]), ph, wait_limit)) {
        s_abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      unsigned char* sEh = smem + st * TC_STAGE_BYTES;
      const uint32_t e0 = smem_u32(sEh), e1 = smem_u32(sEh + TC_EBYTES), t0 = smem_u32(sEh + 2 * TC_EBYTES);
#pragma unroll
      for (int j = 0; j < TC_KS / 8; ++j) {
        const uint64_t ah = smem_desc(e0 + j * (TC_M / 8) * 256);
        const uint64_t al = smem_desc(e1 + j * (TC_M / 8) * 256);
        const uint64_t bh = smem_desc(t0 + j * (N / 8) * 256);
        const uint64_t bl = smem_desc(t0 + N * TC_KS * 4 + j * (N / 8) * 256);
        if constexpr (F16) {
          mma_f16(tmem, ah, bh, idesc, (it > 0 || j > 0) ? 1u : 0u);
          mma_f16(tmem, ah, bl, idesc, 1u);
          mma_f16(tmem, al, bh, idesc, 1u);
        } else {
          mma_tf32(tmem, ah, bh, idesc, (it > 0 || j > 0) ? 1u : 0u);
          if (nprod == 3) {
            mma_tf32(tmem, ah, bl, idesc, 1u);
            mma_tf32(tmem, al, bh, idesc, 1u);
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&bar_r[st]))
                   : "memory");
      committed = it + 1;
    }
    // the last commit arrives once every MMA issued before it has completed
    if (committed > 0) {
      const int last = committed - 1;
      if (!mbar_wait(smem_u32(&bar_r[last % NS]), (last / NS) & 1, wait_limit)) s_abort = 1;
    }
    if (committed < nstage) s_abort = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!s_abort) {
    tc_epilogue<F16>(tmem, warp, lane, smem, s_src, s_dst, s_flg, escale, tscale, tsoff, g, Po, N, nt, D);
  } else if (tid == 0) {
    atomicOr(err, BEM_DEVERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_NMAX));
}

// ------------------------------------------------------- persistent kernel --
// One CTA per SM walks the job list (virtual job v = blockIdx.x + i gridDim.x,
// job v / nchunk, rhs v % nchunk) on one ring of NS stages that runs on
// across job boundaries, with two tensor-memory accumulators so that the
// epilogue of job i overlaps the stages of job i + 1.  Roles (320 threads):
//   warps 0-3  gather producers (as k_grouped_tc_ws; the pair rows of the
//              current job in shared memory, reloaded between jobs behind a
//              named barrier of these four warps);
//   warps 4-7  epilogue: warp w owns tensor-memory lanes 32 (w - 4) .. + 31
//              and runs tc_epilogue's two steps for its 32 pairs through its
//              own shared tile, then releases the accumulator;
//   warp 8     one thread issues the matrix stages' bulk copies;
//   warp 9     one thread issues the MMAs: it waits for an accumulator to be
//              released, runs the job's stages into it, and commits it.
// Every wait is bounded; on expiry the role records the abort and stops, and
// the CTA drains its copies and MMAs before it frees tensor memory.
#define TC_P_THREADS 320
#define TC_P_STAGES 3
#define TC_P_EPI_BYTES (4 * 32 * TC_EPI_STRIDE * 4)
#define TC_P_SMEM (TC_P_STAGES * TC_STAGE_BYTES + TC_P_EPI_BYTES)

template <bool F16, int NS, int LAG>
__global__ void __launch_bounds__(TC_P_THREADS, 1) k_grouped_tc_p(
    const int4* __restrict__ jobs, int njobs, const int* __restrict__ grows, const int* __restrict__ gcols,
    const int64_t* __restrict__ tcoff, const float* __restrict__ tcB, const int* __restrict__ prep_row,
    const int* __restrict__ dst_off, const unsigned char* __restrict__ pflags, const float* __restrict__ prep,
    int row_floats, int nchunk, int rows_per_rhs, float* __restrict__ dst, int64_t exp_stride, int nprod, int kslice,
    int* err, long long wait_limit, int hold_first_copy, const float* __restrict__ escale,
    const float* __restrict__ tscale, const int* __restrict__ tsoff) {
  static_assert(LAG >= 1 && LAG < NS, "the gather lag must leave the MMAs a stage of slack");
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_e[NS], bar_t[NS], bar_r[NS], bar_af[2], bar_ae[2];
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_abort;
  __shared__ int s_src[TC_M];
  constexpr int KSTG = F16 ? 32 : TC_KS;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nvirt = njobs * nchunk;
  // the job of local index i, and its stage count and tile width
  auto job_of = [&](int i, int4& J, int& r, int& nstage, int& N) -> bool {
    const int v = blockIdx.x + i * gridDim.x;
    if (v >= nvirt) return false;
    J = jobs[v / nchunk];
    r = v % nchunk;
    const int g = J.x;
    N = tc_ntile_width(2 * grows[g], J.w);
    const int nks = (2 * gcols[g] + KSTG - 1) / KSTG;
    const int ks0 = (J.z >> 8) * kslice;
    nstage = min(nks, ks0 + kslice) - ks0;
    return true;
  };

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(2 * TC_NMAX));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    s_abort = 0;
    for (int i = 0; i < NS; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_e[i])), "r"(TC_M));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_t[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_r[i])));
    }
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_af[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_ae[i])), "r"(TC_M));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  if (warp < 4) {
    // ---- gather producers ----
    // the job loop is uniform over the four warps (named barriers inside):
    // after an abort the remaining jobs are walked without issuing
    int it = 0, issued = 0;
    int4 J;
    int r, nstage, N;
    for (int i = 0; job_of(i, J, r, nstage, N); ++i) {
      const int p0 = J.y, np = J.z & 255;
      const int ks0 = (J.z >> 8) * kslice;
      asm volatile("bar.sync 1, 128;" ::: "memory");  // every producer is done with the last job's rows
      s_src[tid] = tid < np ? prep_row[p0 + tid] + r * rows_per_rhs : -1;
      asm volatile("bar.sync 1, 128;" ::: "memory");
      for (int k = 0; k < nstage; ++k, ++it) {
        if (s_abort) break;
        const int st = it % NS;
        if (it >= NS && !mbar_wait(smem_u32(&bar_r[st]), ((it / NS) - 1) & 1, wait_limit)) {
          s_abort = 1;
          break;
        }
        unsigned char* sEh = smem + st * TC_STAGE_BYTES;
        unsigned char* sEl = sEh + TC_EBYTES;
        const int ks = ks0 + k;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int item = tid + TC_M * q;
          const int c = ((item >> 5) & 15) * 8 + (item & 7), quad = (item >> 3) & 3, part = item >> 9;
          const int row = s_src[c];
          const float* src = row >= 0
                                 ? prep + (int64_t)row * row_floats + ks * (2 * TC_KS) + part * TC_KS + quad * 4
                                 : prep;
          const uint32_t dsm = smem_u32((part ? sEl : sEh) + core_off(c, quad * 4, TC_M));
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dsm), "l"(src), "r"(row >= 0 ? 16 : 0)
                       : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        ++issued;
        if (it >= LAG) {
          asm volatile("cp.async.wait_group %0;" ::"n"(LAG) : "memory");
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_arrive(smem_u32(&bar_e[(it - LAG) % NS]));
        }
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int j = max(0, issued - LAG); j < issued; ++j) mbar_arrive(smem_u32(&bar_e[j % NS]));
  } else if (warp < 8) {
    // ---- epilogue warps ----
    const int ew = warp - 4;  // tensor-memory lane quarter
    float* tile = (float*)(smem + NS * TC_STAGE_BYTES) + ew * 32 * TC_EPI_STRIDE;
    int4 J;
    int r, nstage, N;
    for (int i = 0;; ++i) {
      // warp-uniform decisions: the tensor-memory loads and shuffles below
      // need all 32 lanes
      const int go = __shfl_sync(0xffffffffu, (!s_abort && job_of(i, J, r, nstage, N)) ? 1 : 0, 0);
      if (!go) break;
      job_of(i, J, r, nstage, N);
      const int a = i & 1;
      int ok = 1;
      if (lane == 0 && !mbar_wait(smem_u32(&bar_af[a]), (i >> 1) & 1, wait_limit)) {
        s_abort = 1;
        ok = 0;
      }
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int g = J.x, p0 = J.y, np = J.z & 255, nt = J.w;
      const int Po = grows[g];
      const float* tsg = F16 ? tscale + tsoff[g] : nullptr;
      float* D = dst + 2 * (int64_t)r * exp_stride;
      // this lane's pair (the row of the tile it fills)
      const int c = 32 * ew + lane;
      const bool pv = c < np;
      const int my_dst = pv ? dst_off[p0 + c] : -1;
      const int my_flg = pv ? (int)pflags[p0 + c] : 0;
      const float my_sc = (F16 && pv) ? escale[prep_row[p0 + c] + r * rows_per_rhs] : 1.f;
      for (int c0 = 0; c0 < N; c0 += 64) {
        const int ncol = min(64, N - c0);
#pragma unroll
        for (int j = 0; j < 64; j += 8) {
          if (j < ncol) {
            uint32_t v[8];
            const uint32_t taddr = tmem + ((uint32_t)(32 * ew) << 16) + (uint32_t)(a * TC_NMAX + c0 + j);
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float* t = tile + lane * TC_EPI_STRIDE + j;
            *(float4*)t = make_float4(__uint_as_float(v[0]), __uint_as_float(v[1]), __uint_as_float(v[2]),
                                      __uint_as_float(v[3]));
            *(float4*)(t + 4) = make_float4(__uint_as_float(v[4]), __uint_as_float(v[5]), __uint_as_float(v[6]),
                                            __uint_as_float(v[7]));
          }
        }
        __syncwarp();
        const int q = (nt * TC_NMAX + c0) / 2 + lane;
        const bool live = 2 * lane < ncol && q < Po;
        int n = (int)sqrtf((float)q);
        if ((n + 1) * (n + 1) <= q) ++n;
        if (n * n > q) --n;
        const int m = q - n * n - n;
        const float ts = (F16 && live) ? tsg[2 * q] : 1.f;
        for (int pc = 0; pc < 32; ++pc) {
          const int dof = __shfl_sync(0xffffffffu, my_dst, pc);
          const int fl = __shfl_sync(0xffffffffu, my_flg, pc);
          const float psc = __shfl_sync(0xffffffffu, my_sc, pc);
          if (dof < 0 || !live) continue;
          const bool neg = ((fl & 1) && (m & 1)) != ((fl & 4) && ((n + m) & 1));
          const bool mflip = ((fl & 1) != 0) != ((fl & 2) != 0);
          float sc = neg ? -1.f : 1.f;
          if (F16) sc *= psc * ts;
          const float2 v = *(const float2*)(tile + pc * TC_EPI_STRIDE + 2 * lane);
          atomicAdd((float2*)(D + 2 * ((int64_t)dof + (mflip ? n * n + n - m : q))),
                    make_float2(sc * v.x, sc * v.y));
        }
        __syncwarp();
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(smem_u32(&bar_ae[a]));
    }
  } else if (warp == 8 && lane == 0) {
    // ---- matrix producer ----
    int it = 0, last = -1;
    int4 J;
    int r, nstage, N;
    for (int i = 0; !s_abort && job_of(i, J, r, nstage, N); ++i) {
      const int g = J.x, nt = J.w;
      const int nks = (2 * gcols[g] + KSTG - 1) / KSTG;
      const int ks0 = (J.z >> 8) * kslice;
      const float* Tg = tcB + tcoff[g] + (int64_t)nt * nks * (2 * TC_NMAX * TC_KS);
      const uint32_t tbytes = (uint32_t)(2 * N * TC_KS * 4);
      for (int k = 0; k < nstage; ++k, ++it) {
        if (s_abort) break;
        const int st = it % NS;
        if (it >= NS && !mbar_wait(smem_u32(&bar_r[st]), ((it / NS) - 1) & 1, wait_limit)) {
          s_abort = 1;
          break;
        }
        if (it == 0 && hold_first_copy) continue;  // diagnostic of the timeout path
        const uint32_t bar = smem_u32(&bar_t[st]);
        unsigned char* sT = smem + st * TC_STAGE_BYTES + 2 * TC_EBYTES;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tbytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_u32(sT)),
                     "l"(Tg + (int64_t)(ks0 + k) * (2 * N * TC_KS)), "r"(tbytes), "r"(bar)
                     : "memory");
        last = it;
      }
    }
    for (int j = max(0, last - NS + 1); j <= last; ++j) {
      if (j == 0 && hold_first_copy) continue;
      if (!mbar_wait(smem_u32(&bar_t[j % NS]), (j / NS) & 1, wait_limit)) s_abort = 1;
    }
  } else if (warp == 9 && lane == 0) {
    // ---- MMA issuer ----
    int it = 0, lastc = -1;  // stage of the last commit
    int4 J;
    int r, nstage, N;
    for (int i = 0; !s_abort && job_of(i, J, r, nstage, N); ++i) {
      const int a = i & 1;
      if (i >= 2 && !mbar_wait(smem_u32(&bar_ae[a]), ((i >> 1) - 1) & 1, wait_limit)) {
        s_abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t idesc = F16 ? instr_desc_f16(N) : instr_desc(N);
      const uint32_t acc = tmem + (uint32_t)(a * TC_NMAX);
      bool done = true;
      for (int k = 0; k < nstage; ++k, ++it) {
        const int st = it % NS;
        const uint32_t ph = (it / NS) & 1;
        if (s_abort || !mbar_wait(smem_u32(&bar_t[st]), ph, wait_limit) ||
            !mbar_wait(smem_u32(&bar_e[st]), ph, wait_limit)) {
          s_abort = 1;
          done = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        unsigned char* sEh = smem + st * TC_STAGE_BYTES;
        const uint32_t e0 = smem_u32(sEh), e1 = smem_u32(sEh + TC_EBYTES), t0 = smem_u32(sEh + 2 * TC_EBYTES);
#pragma unroll
        for (int j = 0; j < TC_KS / 8; ++j) {
          const uint64_t ah = smem_desc(e0 + j * (TC_M / 8) * 256);
          const uint64_t al = smem_desc(e1 + j * (TC_M / 8) * 256);
          const uint64_t bh = smem_desc(t0 + j * (N / 8) * 256);
          const uint64_t bl = smem_desc(t0 + N * TC_KS * 4 + j * (N / 8) * 256);
          if constexpr (F16) {
            mma_f16(acc, ah, bh, idesc, (k > 0 || j > 0) ? 1u : 0u);
            mma_f16(acc, ah, bl, idesc, 1u);
            mma_f16(acc, al, bh, idesc, 1u);
          } else {
            mma_tf32(acc, ah, bh, idesc, (k > 0 || j > 0) ? 1u : 0u);
            if (nprod == 3) {
              mma_tf32(acc, ah, bl, idesc, 1u);
              mma_tf32(acc, al, bh, idesc, 1u);
            }
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&bar_r[st]))
                     : "memory");
        lastc = it;
      }
      if (!done) break;
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&bar_af[a]))
                   : "memory");
    }
    // the last commit arrives once every MMA issued before it has completed
    if (lastc >= 0 && !mbar_wait(smem_u32(&bar_r[lastc % NS]), (lastc / NS) & 1, wait_limit)) s_abort = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (s_abort && tid == 0) atomicOr(err, BEM_DEVERR_TIMEOUT);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_NMAX));
}

// ------------------------------------------------------ source preparation --
// For rhs r0 + rc (rc < nchunk), every box of the source level and every
// reflection f (8), a row of 2 R2 floats: row ((rc * 8 + f) * nbox + b) holds
// s_f(k) M_b[Q_f(k)] as interleaved (re, im), zero-padded to R2, rounded to
// TF32 (hi) plus the remainder (lo), stored per K stage of 16 as
// [hi 16 | lo 16], so that one stage of one pair is 128 contiguous bytes.
#define TC_RHS_CHUNK 4  // right-hand sides per translation launch

__global__ void k_prep(const float* __restrict__ src, int64_t base, int nbox, int P, int R2, int r0, int nchunk,
                       int64_t exp_stride, float* __restrict__ out) {
  // one thread per 4 consecutive floats of a row (one float4 of hi, one of lo)
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per_rhs = (int64_t)8 * nbox;
  const int R4 = R2 / 4;
  if (idx >= nchunk * per_rhs * R4) return;
  const int64_t row = idx / R4;
  const int kr0 = 4 * (int)(idx % R4);
  const int rc = (int)(row / per_rhs);
  const int f = (int)((row % per_rhs) / nbox), b = (int)(row % nbox);
  const float* sb = src + 2 * ((int64_t)(r0 + rc) * exp_stride + base + (int64_t)b * P);
  float v[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int kr = kr0 + e;
    v[e] = 0.f;
    if (kr < 2 * P) {
      bool neg;
      const int ki = reflect_index(kr >> 1, f, &neg);
      v[e] = sb[2 * ki + (kr & 1)];
      if (neg) v[e] = -v[e];
    }
  }
  float4 hi, lo;
  hi.x = tf32_round(v[0]);
  hi.y = tf32_round(v[1]);
  hi.z = tf32_round(v[2]);
  hi.w = tf32_round(v[3]);
  lo = make_float4(v[0] - hi.x, v[1] - hi.y, v[2] - hi.z, v[3] - hi.w);
  float* o = out + row * (2 * (int64_t)R2) + (kr0 / TC_KS) * (2 * TC_KS) + (kr0 % TC_KS);
  *(float4*)o = hi;
  *(float4*)(o + TC_KS) = lo;
}

// FP16 split: one warp per row (rhs r0 + rc, reflection f, box b): row
// (rc * 8 + f) * nbox + b.  The expansion's largest magnitude (reflections
// only permute and negate) picks the power-of-two scale; per K stage of 32
// the row holds [hi 32 | lo 32] halves (128 bytes, as a TF32 stage of 16),
// every lane producing 4 consecutive values of a stage (8-byte stores of hi
// and lo); escale[row] keeps the inverse scale.
__device__ __forceinline__ void prep16_row(const float* __restrict__ src, int64_t base, int nbox, int P, int nks,
                                           int r, int f, int b, int64_t row, int lane, int64_t exp_stride,
                                           float* __restrict__ out, float* __restrict__ escale) {
  const float* sb = src + 2 * ((int64_t)r * exp_stride + base + (int64_t)b * P);
  float m = 0.f;
  for (int kr = lane; kr < 2 * P; kr += 32) m = fmaxf(m, fabsf(sb[kr]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  float sc, iv;
  f16_scale(m, &sc, &iv);
  if (lane == 0) escale[row] = iv;
  const int K = 32 * nks;
  __half* o = (__half*)(out + row * (int64_t)K);
  for (int k4 = 4 * lane; k4 < K; k4 += 128) {
    // values k4 .. k4 + 3: (re, im) of coefficients k4 / 2 and k4 / 2 + 1
    float v[4];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int kc = (k4 >> 1) + e;
      float2 w = make_float2(0.f, 0.f);
      if (kc < P) {
        bool neg;
        const int ki = reflect_index(kc, f, &neg);
        w = *(const float2*)(sb + 2 * ki);
        if (neg) w = make_float2(-w.x, -w.y);
      }
      v[2 * e] = w.x * sc;
      v[2 * e + 1] = w.y * sc;
    }
    __half hi[4], lo[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      hi[e] = __float2half_rn(v[e]);
      lo[e] = __float2half_rn(v[e] - __half2float(hi[e]));
    }
    __half* d = o + (k4 >> 5) * 64 + (k4 & 31);
    *(uint2*)d = *(const uint2*)hi;
    *(uint2*)(d + 32) = *(const uint2*)lo;
  }
}

__global__ void k_prep16(const float* __restrict__ src, int64_t base, int nbox, int P, int nks, int r0, int nchunk,
                         int64_t exp_stride, float* __restrict__ out, float* __restrict__ escale) {
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t per_rhs = (int64_t)8 * nbox;
  if (row >= nchunk * per_rhs) return;
  const int rc = (int)(row / per_rhs);
  const int f = (int)((row % per_rhs) / nbox), b = (int)(row % nbox);
  prep16_row(src, base, nbox, P, nks, r0 + rc, f, b, row, lane, exp_stride, out, escale);
}

// the same for the rows some pair reads (list: rows f * nbox + b of one rhs),
// when the operator's pairs use few of the 8 reflections of each box (M2M:
// every child box is read once, with the reflection of its octant)
__global__ void k_prep16_list(const float* __restrict__ src, int64_t base, int nbox, int P, int nks, int r0,
                              int nchunk, const int* __restrict__ list, int nlist, int64_t exp_stride,
                              float* __restrict__ out, float* __restrict__ escale) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (int64_t)nchunk * nlist) return;
  const int rc = (int)(w / nlist);
  const int lr = list[w % nlist];
  const int f = lr / nbox, b = lr % nbox;
  prep16_row(src, base, nbox, P, nks, r0 + rc, f, b, (int64_t)rc * 8 * nbox + lr, lane, exp_stride, out, escale);
}

__global__ void k_prep_rows(int np, const int* __restrict__ src_off, const unsigned char* __restrict__ flags,
                            int64_t base, int P, int nbox, int* rows) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  int b = (int)((src_off[i] - base) / P);
  rows[i] = (int)flags[i] * nbox + b;
}

// -------------------------------------------------------------------- host --

// K per stage of the handle's translation form: 32 (FP16 split) or 16 (TF32)
static inline int tc_kstage(const bem_handle* h) { return h->tc_fp16 ? 32 : TC_KS; }
// floats per prepared source row: stages x 32 floats (hi and lo, 128 bytes)
static inline int prep_row_floats(const bem_handle* h, int P) {
  const int ks = tc_kstage(h);
  return ((2 * P + ks - 1) / ks) * 2 * TC_KS;
}

int bem_build_tc(bem_handle* h, GroupedOp& op, int src_level, cudaStream_t s) {
  if (op.ngroups == 0) return BEM_OK;
  op.src_level = src_level;
  const int KSTG = tc_kstage(h);
  {
    LevelInfo& sl = h->lev[src_level];
    const int chunk = std::min(h->nrhs_max, TC_RHS_CHUNK);
    const int64_t rows = (int64_t)chunk * 8 * sl.nbox;
    int64_t need = rows * prep_row_floats(h, sl.P);
    if (need > h->prep_len) {
      float* p;
      BEM_TRY(bem_alloc(h, &p, need));  // grows monotonically; older buffers stay in the handle's list
      h->prep = p;
      h->prep_len = need;
    }
    if (h->tc_fp16 && rows > h->prep_scale_len) {
      float* p;
      BEM_TRY(bem_alloc(h, &p, rows));
      h->prep_scale = p;
      h->prep_scale_len = rows;
    }
    BEM_TRY(bem_alloc(h, &op.d_prep_row, std::max(op.npairs, 1)));
    if (op.npairs > 0)
      k_prep_rows<<<(op.npairs + 255) / 256, 256, 0, s>>>(op.npairs, op.d_src_off, op.d_flags, sl.exp_base, sl.P,
                                                          sl.nbox, op.d_prep_row);
    BEM_CUDA(cudaGetLastError());
    // the rows the pairs read: when they are under half of all 8 nbox rows,
    // the FP16 preparation runs over their list alone
    if (h->tc_fp16 && op.npairs > 0) {
      std::vector<int> pr(op.npairs);
      BEM_CUDA(cudaMemcpyAsync(pr.data(), op.d_prep_row, op.npairs * sizeof(int), cudaMemcpyDeviceToHost, s));
      BEM_CUDA(cudaStreamSynchronize(s));
      std::sort(pr.begin(), pr.end());
      pr.erase(std::unique(pr.begin(), pr.end()), pr.end());
      if (2 * (int64_t)pr.size() < (int64_t)8 * sl.nbox) {
        op.n_prep_list = (int)pr.size();
        BEM_TRY(bem_alloc(h, &op.d_prep_list, pr.size()));
        BEM_CUDA(cudaMemcpyAsync(op.d_prep_list, pr.data(), pr.size() * sizeof(int), cudaMemcpyHostToDevice, s));
      }
    }
  }
  BEM_CUDA(cudaFuncSetAttribute(k_grouped_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  BEM_CUDA(cudaFuncSetAttribute(k_grouped_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  BEM_CUDA(cudaFuncSetAttribute(k_grouped_tc_ws<false, 4, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                4 * TC_STAGE_BYTES));
  BEM_CUDA(cudaFuncSetAttribute(k_grouped_tc_ws<true, 4, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                4 * TC_STAGE_BYTES));
  BEM_CUDA(cudaFuncSetAttribute(k_grouped_tc_ws<false, 2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                2 * TC_STAGE_BYTES));
  BEM_CUDA(cudaFuncSetAttribute(k_grouped_tc_ws<true, 2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                2 * TC_STAGE_BYTES));
  BEM_CUDA(cudaFuncSetAttribute(k_grouped_tc_p<false, TC_P_STAGES, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                TC_P_SMEM));
  BEM_CUDA(cudaFuncSetAttribute(k_grouped_tc_p<true, TC_P_STAGES, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                TC_P_SMEM));
  std::vector<int64_t> off(op.ngroups);
  std::vector<int> toff(op.ngroups);
  int64_t tot = 0;
  int ttot = 0;
  for (int g = 0; g < op.ngroups; ++g) {
    int nnt = (2 * op.rows[g] + TC_NMAX - 1) / TC_NMAX, nks = (2 * op.cols[g] + KSTG - 1) / KSTG;
    off[g] = tot;
    tot += (int64_t)nnt * nks * 2 * TC_NMAX * TC_KS;
    toff[g] = ttot;
    ttot += 2 * op.rows[g];
  }
  BEM_TRY(bem_alloc(h, &op.tcA, std::max<int64_t>(tot, 4)));
  float* rsc = nullptr;
  if (h->tc_fp16) {
    BEM_TRY(bem_alloc(h, &op.tscale, std::max(ttot, 1)));
    BEM_TRY(bem_alloc(h, &op.d_tsoff, op.ngroups));
    BEM_CUDA(cudaMemcpyAsync(op.d_tsoff, toff.data(), toff.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMallocAsync((void**)&rsc, std::max(ttot, 1) * sizeof(float), s));
  }
  for (int g = 0; g < op.ngroups; ++g) {
    int nnt = (2 * op.rows[g] + TC_NMAX - 1) / TC_NMAX, nks = (2 * op.cols[g] + KSTG - 1) / KSTG;
    const float* T = (const float*)op.mats_base + 2 * op.mat_off[g];
    if (h->tc_fp16) {
      k_tc_rowscale<<<(op.rows[g] + 7) / 8, 256, 0, s>>>(T, op.rows[g], op.cols[g], rsc + toff[g],
                                                          op.tscale + toff[g]);
      k_tc_pack16<<<nnt * nks, 256, 0, s>>>(T, op.rows[g], op.cols[g], nks, rsc + toff[g], op.tcA + off[g]);
    } else {
      k_tc_pack<<<nnt * nks, 256, 0, s>>>(T, op.rows[g], op.cols[g], nks, nnt, op.tcA + off[g]);
    }
    BEM_CUDA(cudaGetLastError());
  }
  if (rsc) BEM_CUDA(cudaFreeAsync(rsc, s));
  // K stages per job: TC_KSLICE.  When the operator has too few (pair tile,
  // row tile) jobs to give every SM two CTAs, a second job list with shorter
  // slices (down to 2 stages) lets the small translations (M2M, L2L, the
  // upper M2L levels) spread their stage-by-stage latency over more CTAs; only
  // single-rhs launches use it.
  int64_t base = 0;
  int nks_max = 1;
  for (int g = 0; g < op.ngroups; ++g) {
    int np = op.pair_start[g + 1] - op.pair_start[g];
    base += (int64_t)((np + TC_M - 1) / TC_M) * ((2 * op.rows[g] + TC_NMAX - 1) / TC_NMAX);
    nks_max = std::max(nks_max, (2 * op.cols[g] + KSTG - 1) / KSTG);
  }
  int nsm = 0;
  BEM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
  op.tc_want = 2 * (int64_t)std::max(nsm, 1);
  const int kmax = std::min(TC_KSLICE, std::max(2, h->tc_kslice_max));
  int ksplit = kmax;
  // (FP16 stages hold twice the K of TF32 ones, so their shortest slice is one stage)
  const int kmin = h->tc_fp16 ? 1 : 2;
  if (base > 0 && base * ((nks_max + kmax - 1) / kmax) < op.tc_want) {
    const int64_t slices = (op.tc_want + base - 1) / base;
    ksplit = (int)std::max<int64_t>(kmin, std::min<int64_t>(kmax, (nks_max + slices - 1) / slices));
  }
  auto make_jobs = [&](int kslice) {
    std::vector<int4> js;
    for (int g = 0; g < op.ngroups; ++g) {
      int np = op.pair_start[g + 1] - op.pair_start[g];
      int nnt = (2 * op.rows[g] + TC_NMAX - 1) / TC_NMAX;
      int nks = (2 * op.cols[g] + KSTG - 1) / KSTG;
      for (int p0 = 0; p0 < np; p0 += TC_M)
        for (int nt = 0; nt < nnt; ++nt)
          for (int sl = 0; sl * kslice < nks; ++sl)
            js.push_back(make_int4(g, op.pair_start[g] + p0, std::min(TC_M, np - p0) | (sl << 8), nt));
    }
    return js;
  };
  std::vector<int4> jobs = make_jobs(kmax);
  op.tc_kslice = kmax;
  if (ksplit < kmax) {
    std::vector<int4> js = make_jobs(ksplit);
    op.tc_kslice_split = ksplit;
    op.n_tc_jobs_split = (int)js.size();
    BEM_TRY(bem_alloc(h, &op.d_tc_jobs_split, js.size()));
    BEM_CUDA(cudaMemcpyAsync(op.d_tc_jobs_split, js.data(), js.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
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
  LevelInfo& sl = h->lev[op.src_level];
  const int row_floats = prep_row_floats(h, sl.P);
  const int chunk = std::min(h->nrhs_max, TC_RHS_CHUNK);
  for (int r0 = 0; r0 < nrhs; r0 += chunk) {
    // up to `chunk` right-hand sides per launch share each matrix stage via L2
    const int nc = std::min(chunk, nrhs - r0);
    if (h->tc_fp16 && op.n_prep_list > 0) {
      const int64_t rows = (int64_t)nc * op.n_prep_list;
      k_prep16_list<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(
          (const float*)src, sl.exp_base, sl.nbox, sl.P, row_floats / (2 * TC_KS), r0, nc, op.d_prep_list,
          op.n_prep_list, h->exp_total, h->prep, h->prep_scale);
    } else if (h->tc_fp16) {
      const int64_t rows = (int64_t)nc * 8 * sl.nbox;
      k_prep16<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(
          (const float*)src, sl.exp_base, sl.nbox, sl.P, row_floats / (2 * TC_KS), r0, nc, h->exp_total, h->prep,
          h->prep_scale);
    } else {
      const int R2 = row_floats / 2;
      const int64_t n = (int64_t)nc * 8 * sl.nbox * (R2 / 4);
      k_prep<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const float*)src, sl.exp_base, sl.nbox, sl.P, R2, r0, nc,
                                                          h->exp_total, h->prep);
    }
    BEM_CUDA(cudaGetLastError());
    // one right-hand side and too few CTAs for the SMs: the job list with
    // shorter K slices (with 2-4 right-hand sides per launch the extra
    // slices' atomics cost more than the added CTAs give back)
    const bool split = nc == 1 && op.n_tc_jobs_split > 0;
    // the loop: the handle's choice, or per operator (measured: the persistent
    // kernel on the few long M2M jobs, two warp-specialised stages elsewhere)
    const int pipe = h->tc_pipeline > 0 ? h->tc_pipeline : (op.upward ? 3 : 2);
    if (pipe == 3) {
      // persistent: one CTA per SM walks the job list
      const int njobs = split ? op.n_tc_jobs_split : op.n_tc_jobs;
      const int grid = (int)std::min<int64_t>((int64_t)njobs * nc, std::max(h->nsm, 1));
      auto pk = h->tc_fp16 ? k_grouped_tc_p<true, TC_P_STAGES, 1> : k_grouped_tc_p<false, TC_P_STAGES, 1>;
      pk<<<grid, TC_P_THREADS, TC_P_SMEM, s>>>(
          split ? op.d_tc_jobs_split : op.d_tc_jobs, njobs, op.d_group_rows, op.d_group_cols, op.d_tc_off, op.tcA,
          op.d_prep_row, op.d_dst_off, op.d_flags, h->prep, row_floats, nc, 8 * sl.nbox,
          (float*)dst + 2 * (int64_t)r0 * h->exp_total, h->exp_total, h->mode == BEM_MODE_FMM_TF32 ? 1 : 3,
          split ? op.tc_kslice_split : op.tc_kslice, h->d_err, h->tc_wait_limit, h->tc_hold_first_copy,
          h->prep_scale, op.tscale, op.d_tsoff);
      BEM_CUDA(cudaGetLastError());
      *launches += 2;
      continue;
    }
    // tc_pipeline: 1 block-synchronous two-stage loop, 2 / 4 warp-specialised with 2 / 4 stages
    auto kern = pipe == 4   ? (h->tc_fp16 ? k_grouped_tc_ws<true, 4, 2> : k_grouped_tc_ws<false, 4, 2>)
                : pipe == 2 ? (h->tc_fp16 ? k_grouped_tc_ws<true, 2, 1> : k_grouped_tc_ws<false, 2, 1>)
                            : (h->tc_fp16 ? k_grouped_tc<true> : k_grouped_tc<false>);
    const size_t smem = pipe == 4 ? 4 * TC_STAGE_BYTES : 2 * TC_STAGE_BYTES;
    kern<<<(split ? op.n_tc_jobs_split : op.n_tc_jobs) * nc, TC_THREADS, smem, s>>>(
        split ? op.d_tc_jobs_split : op.d_tc_jobs, op.d_group_rows, op.d_group_cols, op.d_tc_off, op.tcA,
        op.d_prep_row, op.d_dst_off, op.d_flags, h->prep, row_floats, nc, 8 * sl.nbox,
        (float*)dst + 2 * (int64_t)r0 * h->exp_total, h->exp_total, h->mode == BEM_MODE_FMM_TF32 ? 1 : 3,
        split ? op.tc_kslice_split : op.tc_kslice, h->d_err, h->tc_wait_limit, h->tc_hold_first_copy,
        h->prep_scale, op.tscale, op.d_tsoff);
    BEM_CUDA(cudaGetLastError());
    *launches += 2;
  }
  return BEM_OK;
}

// ------------------------------------------------------ peak microbenchmarks --
// Roofline denominators that no driver measurement covers: the dense TF32
// tensor rate of tcgen05 (the translations' 3xTF32 runs three products per
// algorithmic flop) and the FP32 rate of packed f32x2 FMAs (the P2P's pipe).

// Every CTA issues `iters` back-to-back M = 128, N = 256, K = 8 TF32 MMAs
// from one thread into one TMEM accumulator, with both operands resident in
// shared memory, then commits once and waits (bounded) for completion.
template <bool F16>
__global__ void __launch_bounds__(128, 1) k_peak_tc(int iters, int* err, float* sink) {
  __shared__ __align__(1024) unsigned char ops[TC_M * 8 * 4 + TC_NMAX * 8 * 4];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_ok;
  const int tid = threadIdx.x, warp = tid >> 5;
  if constexpr (F16) {
    for (int i = tid; i < (int)(sizeof(ops) / 2); i += blockDim.x) ((__half*)ops)[i] = __float2half_rn(1.0f + 1e-3f * (i & 7));
  } else {
    for (int i = tid; i < (int)(sizeof(ops) / 4); i += blockDim.x) ((float*)ops)[i] = tf32_round(1.0f + 1e-3f * (i & 7));
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(TC_NMAX));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // operands written by threads, read by the MMA
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  bool ok = true;
  if (tid == 0) {
    const uint64_t a = smem_desc(smem_u32(ops)), b = smem_desc(smem_u32(ops + TC_M * 8 * 4));
    const uint32_t idesc = F16 ? instr_desc_f16(TC_NMAX) : instr_desc(TC_NMAX);
    for (int i = 0; i < iters; ++i) {
      if constexpr (F16)
        mma_f16(tmem, a, b, idesc, i > 0 ? 1u : 0u);
      else
        mma_tf32(tmem, a, b, idesc, i > 0 ? 1u : 0u);
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&bar))
                 : "memory");
    ok = mbar_wait(smem_u32(&bar), 0);
    if (!ok) atomicOr(err, BEM_DEVERR_TIMEOUT);
    s_ok = ok ? 1 : 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) {  // one accumulator value leaves the kernel, so the work cannot be dropped
    uint32_t v;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(v) : "r"(tmem) : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (tid == 0 && s_ok) sink[blockIdx.x] = __uint_as_float(v);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_NMAX));
}

// Every thread runs 8 independent chains of packed f32x2 FMAs (4 flops each).
__global__ void __launch_bounds__(256) k_peak_fp32(int iters, float* sink) {
  unsigned long long acc[8];
  const float s = 1.0f + 1e-7f * threadIdx.x;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float v = s + j;
    asm("mov.b64 %0, {%1, %2};" : "=l"(acc[j]) : "f"(v), "f"(v));
  }
  unsigned long long m, c;
  asm("mov.b64 %0, {%1, %2};" : "=l"(m) : "f"(0.9999999f), "f"(0.9999999f));
  asm("mov.b64 %0, {%1, %2};" : "=l"(c) : "f"(1e-7f), "f"(1e-7f));
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(acc[j]) : "l"(m), "l"(c));
  }
  float t = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(acc[j]));
    t += lo + hi;
  }
  if (t == 12345.f) sink[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

extern "C" int bem_peak_probe(int which, int iters, double* tflops, void* stream) {
  bem_set_error("");
  if (!tflops || iters < 1 || iters > (1 << 20) || which < 0 || which > 2)
    return bem_fail(BEM_ERR_INVALID_ARG,
                    "which must be 0 (FP32), 1 (TF32) or 2 (FP16), 1 <= iters <= 2^20, tflops non-NULL");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  BEM_CUDA(cudaGetDevice(&dev));
  BEM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = which >= 1 ? 2 * nsm : 8 * nsm, threads = which >= 1 ? 128 : 256;
  float* sink = nullptr;
  int* err = nullptr;
  BEM_CUDA(cudaMallocAsync((void**)&sink, sizeof(float) * blocks * threads, s));
  BEM_CUDA(cudaMallocAsync((void**)&err, sizeof(int), s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = BEM_OK;
  float ms = 0.f;
  int herr = 0;
  auto run = [&]() -> int {
    BEM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up, the second is timed
      BEM_CUDA(cudaEventRecord(e0, s));
      if (which == 1)
        k_peak_tc<false><<<blocks, threads, 0, s>>>(iters, err, sink);
      else if (which == 2)
        k_peak_tc<true><<<blocks, threads, 0, s>>>(iters, err, sink);
      else
        k_peak_fp32<<<blocks, threads, 0, s>>>(iters, sink);
      BEM_CUDA(cudaGetLastError());
      BEM_CUDA(cudaEventRecord(e1, s));
    }
    BEM_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    BEM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    return BEM_OK;
  };
  rc = run();
  cudaFreeAsync(sink, s);
  cudaFreeAsync(err, s);
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != BEM_OK) return rc;
  if (herr) return bem_fail(BEM_ERR_TIMEOUT, "a bounded wait of the tensor-core probe expired");
  const double flops = which == 1   ? (double)blocks * iters * 2.0 * TC_M * TC_NMAX * 8
                      : which == 2 ? (double)blocks * iters * 2.0 * TC_M * TC_NMAX * 16
                                   : (double)blocks * threads * iters * 8 * 4;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return BEM_OK;
}
