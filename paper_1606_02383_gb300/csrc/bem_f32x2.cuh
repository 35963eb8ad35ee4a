// bem_f32x2.cuh -- packed FP32 pairs (Blackwell f32x2 instructions): one lane
// evaluates the same source point for two targets in one instruction per
// operation.  Shared by the forward and the transposed near-field kernels.
#pragma once

typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk2(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk2(f32x2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
// -a: both sign bits flipped by an integer xor (ALU pipe, not the FMA pipe)
__device__ __forceinline__ f32x2 neg2(f32x2 a) {
  f32x2 r;
  asm("xor.b64 %0, %1, 0x8000000080000000;" : "=l"(r) : "l"(a));
  return r;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) { return add2(a, neg2(b)); }
