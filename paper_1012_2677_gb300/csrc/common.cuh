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

// The energy record of one state, by one block (blockDim.x a multiple of 32): pe and virial from the
// force kernel's per-block partials pv (scaled by pe_scale: 1/2 for a full list, where every pair
// is visited twice), ke from the integrator's partials kp, each summed in a fixed order; thread 0
// writes energies[0..3] = (pe, ke, virial, step) and appends (step, pe, ke, vir) to the log if there
// is room.  The partials are read past L1 (they may have been written by other blocks of the same
// launch).
__device__ __forceinline__ void energy_record_block(const double* pv, int nbf, const double* kp, int nbi,
                                                    double pe_scale, double* energies, double* log, int64_t cap,
                                                    int64_t* count, double step) {
  double pe = 0.0, vir = 0.0, ke = 0.0;
  for (int b = threadIdx.x; b < nbf; b += blockDim.x) {
    pe += __ldcg(pv + 2 * (size_t)b);
    vir += __ldcg(pv + 2 * (size_t)b + 1);
  }
  for (int b = threadIdx.x; b < nbi; b += blockDim.x) ke += __ldcg(kp + b);
  // the three sums side by side (each in block_sum's order: warp butterflies, then warp 0)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    pe += __shfl_xor_sync(0xffffffffu, pe, o);
    vir += __shfl_xor_sync(0xffffffffu, vir, o);
    ke += __shfl_xor_sync(0xffffffffu, ke, o);
  }
  __shared__ double sh3[3][32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) {
    sh3[0][w] = pe;
    sh3[1][w] = vir;
    sh3[2][w] = ke;
  }
  __syncthreads();
  if (w == 0) {
    const bool in = l < (int)(blockDim.x >> 5);
    pe = in ? sh3[0][l] : 0.0;
    vir = in ? sh3[1][l] : 0.0;
    ke = in ? sh3[2][l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      pe += __shfl_xor_sync(0xffffffffu, pe, o);
      vir += __shfl_xor_sync(0xffffffffu, vir, o);
      ke += __shfl_xor_sync(0xffffffffu, ke, o);
    }
  }
  if (threadIdx.x == 0) {
    pe *= pe_scale;
    vir *= pe_scale;
    energies[0] = pe;
    energies[1] = ke;
    energies[2] = vir;
    energies[3] = step;
    if (log != nullptr) {
      const int64_t k = *count;
      if (k < cap) {
        log[4 * k + 0] = step;
        log[4 * k + 1] = pe;
        log[4 * k + 2] = ke;
        log[4 * k + 3] = vir;
      }
      *count = k + 1;
    }
  }
}

__device__ __forceinline__ bool finite_d(double v) {
  return (__double_as_longlong(v) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}

__device__ __forceinline__ bool finite_f(float v) {
  return (__float_as_int(v) & 0x7f800000) != 0x7f800000;
}

// Format conversions between binary32 and binary64 with integer operations only, so that they
// take no slots of the FP64 pipe (2 operations per clock per SM on this part).  From the IEEE 754
// layouts: binary32 has an 8-bit exponent with bias 127 and 23 stored mantissa bits, binary64 an
// 11-bit exponent with bias 1023 and 52 stored mantissa bits.
//
// f32_to_f64: exact.  Zero keeps its sign; binary32 subnormals (below 1.2e-38) become zero of the
// same sign; infinities and NaNs map to infinities and NaNs.
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned int u = (unsigned int)__float_as_int(f);
  const unsigned int e = (u >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  unsigned long long bits = sign;
  if (e == 0xffu) bits |= 0x7ff0000000000000ULL | ((unsigned long long)(u & 0x7fffffu) << 29);
  else if (e != 0u) bits |= ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}

// f64_to_f32: rounded to nearest (ties away from zero) at the 24th significant bit.  Magnitudes
// below 2^-126 give zero of the same sign, magnitudes that round to 2^128 or more give infinity;
// infinities and NaNs map to infinities and NaNs.
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0x7ff) return __int_as_float((int)(sign | 0x7f800000u | (unsigned int)((b >> 29) & 0x7fffffu) |
                                              ((b & 0xfffffffffffffULL) ? 0x400000u : 0u)));
  if (e < 1023 - 126) return __int_as_float((int)sign);
  // exponent and top 23 mantissa bits, plus the rounding bit (bit 28); a carry into the exponent
  // is the correct result (and gives infinity past the largest binary32)
  unsigned int r = ((unsigned int)(e - 896) << 23) + (unsigned int)((b >> 29) & 0x7fffffu) +
                   (unsigned int)((b >> 28) & 1u);
  if (e - 896 >= 0xff || r >= 0x7f800000u) r = 0x7f800000u;
  return __int_as_float((int)(sign | r));
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

// Fixed-point coordinate of a stored FP64 coordinate x_state (positive, normal): round(x_state 2^qk)
// mod 2^32, from the FP64 bits with integer operations only.  x_state = m 2^(e - 52) with the
// 53-bit significand m, so x_state 2^qk = m 2^(e + qk - 52); the kernels keep 52 - e - qk in
// [1, 63] (qk <= 40 and stored coordinates in [2, 2^11)), so the value is m shifted right with
// rounding half up.
__device__ __forceinline__ uint32_t fixq(double xs, int qk) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(xs);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  const unsigned long long m = (b & 0xfffffffffffffULL) | (1ULL << 52);
  const int sh = 52 - e - qk;
  if (sh <= 0) return (uint32_t)(m << (-sh < 63 ? -sh : 63));
  if (sh >= 64) return 0u;
  return (uint32_t)((m + (1ULL << (sh - 1))) >> sh);
}

// Difference of two fixed-point coordinates as an FP32 number of units u (one rounding, to 24
// significant bits; the integer difference itself is exact modulo 2^32).
__device__ __forceinline__ float qdiff(uint32_t a, uint32_t b) { return __int2float_rn((int)(a - b)); }

// ---- asynchronous bulk copies into shared memory (cp.async.bulk + mbarrier, sm_90 and later) ----
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Loads from 32-bit shared-memory addresses (the pair loops index staged arrays this way, so the
// address arithmetic stays 32-bit).  Volatile keeps them ordered with the CTA barriers around
// the staging of the next tile into the same bytes.
__device__ __forceinline__ float4 lds_f4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ uint4 lds_u4(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ uint32_t lds_u16(uint32_t a) {
  unsigned short v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ int lds_s32(uint32_t a) {
  int v;
  asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Order this thread's earlier shared-memory accesses before later bulk-copy (async proxy) writes.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// One arrival on the barrier announcing `bytes` of bulk-copy data for the current phase.
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// Bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16), completing on bar.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// Cell labelling without the FP64 pipe beyond the subtraction and the product.  cmp_ge_d: a >= b
// for a finite FP64 value b > 0 (the two's-complement order of the bit patterns matches the FP64
// order there; a NaN compares as at least b).  floor_to_int: floor(t) for 0 <= t < 2^31 from the bit
// pattern (mantissa shifted by the exponent), -1 for any t < 0 (also -0) and INT_MAX for t >= 2^31,
// infinities and NaN: the callers clamp to [0, n - 1], where these agree with floor.
__device__ __forceinline__ bool cmp_ge_d(double a, double b) {
  return __double_as_longlong(a) >= __double_as_longlong(b);
}
__device__ __forceinline__ int floor_to_int(double t) {
  const long long b = __double_as_longlong(t);
  if (b < 0) return -1;
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  if (e < 0) return 0;
  if (e > 30) return 0x7fffffff;
  const unsigned long long m = ((unsigned long long)b & 0xfffffffffffffULL) | 0x10000000000000ULL;
  return (int)(m >> (52 - e));
}

// 4-byte asynchronous copy global -> shared (cp.async, no register staging); the issuing thread's
// copies have landed after cp_async_wait_all.
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// try_wait with a suspend-time hint: the thread may sleep up to `hint_ns` nanoseconds inside the
// instruction until the phase completes, instead of spinning on issue slots.
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity, uint32_t hint_ns = 1000000u) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return r != 0;
}

constexpr long long kWaitBudget = 4000000000LL;  // ~2 s at 2 GHz: a wait that long means a fault

// Wait for phase `parity` of bar to complete, giving up after `budget` clock cycles (false).  A
// budget below the default also drops the suspend hint, so that a short budget is not outlasted
// by one suspended try_wait.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long budget) {
  const uint32_t hint = budget < kWaitBudget ? 0u : 1000000u;
  const long long t0 = clock64();
  while (!mbar_test(bar, parity, hint))
    if (clock64() - t0 > budget) return false;
  return true;
}

}  // namespace ljmd
