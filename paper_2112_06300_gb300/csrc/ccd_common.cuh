// Device helpers shared by the broad- and narrow-phase kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ccd {

constexpr int kWarp = 32;

// Order-preserving map of a float to uint32 (radix-sort key): negative values
// are bit-inverted, non-negative ones get the sign bit set.
__device__ __forceinline__ uint32_t f32_sort_key(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Order-preserving map of a finite double to int64 with -0 mapped to +0, so
// that signed integer comparison equals numeric comparison.  Lets the exact
// FP64 box tests and min/max run on the integer pipes, not the FP64 units.
__device__ __forceinline__ long long f64_ord(double d) {
  long long s = __double_as_longlong(d);
  s = (s == (long long)0x8000000000000000ull) ? 0ll : s;
  return s >= 0 ? s : (s ^ 0x7FFFFFFFFFFFFFFFll);
}

__device__ __forceinline__ double dmin_int(double a, double b) {
  return f64_ord(a) <= f64_ord(b) ? a : b;
}
__device__ __forceinline__ double dmax_int(double a, double b) {
  return f64_ord(a) >= f64_ord(b) ? a : b;
}

// |d| and max of non-negative doubles by bit manipulation.
__device__ __forceinline__ double dabs_int(double d) {
  return __longlong_as_double(__double_as_longlong(d) & 0x7FFFFFFFFFFFFFFFll);
}

// n / 2^l as a double, exact for n <= 2^53 and l <= 53, assembled from bits.
__device__ __forceinline__ double dyadic(uint64_t n, int l) {
  if (n == 0) return 0.0;
  int msb = 63 - __clzll((long long)n);
  uint64_t frac = msb <= 52 ? (n << (52 - msb)) : (n >> (msb - 52));
  frac &= 0x000FFFFFFFFFFFFFull;
  uint64_t exp = (uint64_t)(msb - l + 1023);
  return __longlong_as_double((long long)((exp << 52) | frac));
}

// Lane-aggregated atomic add: one atomic per warp for all active lanes with
// pred set; returns this lane's offset.
__device__ __forceinline__ unsigned long long warp_append(unsigned long long *ctr, bool pred,
                                                          unsigned mask) {
  unsigned ballot = __ballot_sync(mask, pred);
  unsigned long long base = 0;
  int leader = __ffs(mask) - 1;
  int lane = threadIdx.x & 31;
  if (lane == leader && ballot) base = atomicAdd(ctr, (unsigned long long)__popc(ballot));
  base = __shfl_sync(mask, base, leader);
  return base + __popc(ballot & ((1u << lane) - 1u));
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

}  // namespace ccd
