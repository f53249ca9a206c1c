// Device helpers shared by the kernels of libljmd.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ljmd_internal.h"

namespace ljmd {

__host__ __device__ __forceinline__ dvec4 make_dvec4(double a, double b, double c, double d) {
  dvec4 r;
  r.x = a;
  r.y = b;
  r.z = c;
  r.w = d;
  return r;
}

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

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum of a per-thread double over the block (blockDim.x a multiple of 32, <= 1024).
// Fixed order: warp butterflies, then warp 0 sums the warp totals.  Result in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

__device__ __forceinline__ float block_max(float v, float* sh) {
  v = warp_max(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  float t = 0.0f;
  if (w == 0) {
    t = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0f;
    t = warp_max(t);
  }
  return t;
}

__device__ __forceinline__ bool finite_d(double v) {
  return (__double_as_longlong(v) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}

__device__ __forceinline__ bool finite_f(float v) {
  return (__float_as_int(v) & 0x7f800000) != 0x7f800000;
}

// FP32 split of a stored coordinate x_state in [2^(p-1), 2^(p+1)):
// hi = x_state truncated to 24 significant bits (exact as a float),
// lo = x_state - hi rounded to FP32.  Integer operations only (no FP64 pipe):
// hi keeps the sign, exponent and top 23 stored mantissa bits; lo is the
// remaining 29 mantissa bits times 2^(e - 52).
__device__ __forceinline__ void split_hi_lo(double xs, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(xs);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  const unsigned int sign = (unsigned int)(b >> 63) << 31;
  const unsigned int mhi = (unsigned int)((b >> 29) & 0x7fffffu);
  hi = __int_as_float((int)(sign | ((unsigned int)(e + 127) << 23) | mhi));
  const unsigned int mlo = (unsigned int)(b & 0x1fffffffu);
  const float scale = __int_as_float((e - 52 + 127) << 23);  // 2^(e-52), normal for e >= -74
  lo = __uint2float_rn(mlo) * scale;
  if (sign) lo = -lo;
}

}  // namespace ljmd
