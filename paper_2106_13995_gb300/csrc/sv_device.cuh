// Device helpers: complex arithmetic on interleaved float2/double2 and index
// bit manipulation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sv {

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

__device__ __forceinline__ float2 cmake(float r, float i) { return make_float2(r, i); }
__device__ __forceinline__ double2 cmake(double r, double i) { return make_double2(r, i); }

// acc + a * b
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C z;
  z.x = a.x * b.x - a.y * b.y;
  z.y = a.x * b.y + a.y * b.x;
  return z;
}
template <typename C> __device__ __forceinline__ C czero() {
  C z;
  z.x = 0;
  z.y = 0;
  return z;
}

// Insert a zero bit at position p (bits at >= p move up by one).
__device__ __forceinline__ uint64_t ins0(uint64_t x, int p) {
  const uint64_t lo = x & ((1ull << p) - 1);
  return ((x ^ lo) << 1) | lo;
}
__device__ __forceinline__ uint32_t ins0(uint32_t x, int p) {
  const uint32_t lo = x & ((1u << p) - 1);
  return ((x ^ lo) << 1) | lo;
}

// Insert zero bits at every set position of `fixed`, lowest first.
__device__ __forceinline__ uint32_t ins0_mask(uint32_t x, uint32_t fixed) {
  while (fixed) {
    const int p = __ffs(fixed) - 1;
    fixed &= fixed - 1;
    x = ins0(x, p);
  }
  return x;
}
__device__ __forceinline__ uint64_t ins0_mask64(uint64_t x, uint64_t fixed) {
  while (fixed) {
    const int p = __ffsll((long long)fixed) - 1;
    fixed &= fixed - 1;
    x = ins0(x, p);
  }
  return x;
}

// FP64 warp sum.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

}  // namespace sv
