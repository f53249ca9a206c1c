// Force over the sorted pair list (Alg. 4 with Alg. 5's branch-free cutoff and Alg. 6's
// explicit expression).  A group of LANES threads owns one key particle i: the lanes stride
// through i's partners (coalesced SortedList reads), keep q_i and the partial f_i in
// registers, and reduce f_i with shuffles at the end of the row.
//
//   pair coefficient  f = ri2 s3i (24 eps - 48 eps s3i) + 8 eps c2 / sigma^2,
//                     ri2 = 1 / r^2, s3i = (sigma^2 ri2)^3          (Alg. 6 in eps, sigma units)
//   force on i        f (q_j - q_i), zero for r^2 >= r_c^2 (select, no branch; Alg. 5)
//   energy            V = 4 eps [s3i (s3i - 1) + c2 r^2 / sigma^2 + c0]   (Eq. 2)
//   virial            -f r^2   (= r_ij . F_ij)
//
// LJ_LIST_FULL: every pair is visited from both ends; f_i is written once, no atomics, and
//               the result does not depend on scheduling.  Energies are halved at the end.
// LJ_LIST_HALF: key = lower index (Sec. 2.4); the partner's reaction -f (q_j - q_i) is
//               scattered with atomics (Newton's third law), so F must be zeroed first.
//
// Mixed form: q_j - q_i from the hi/lo FP32 split of the stored coordinates (exact hi
// difference, one rounding overall), FP32 pair arithmetic and accumulation per row, FP64
// per-thread and per-block energy sums.  FP64 form: everything in FP64.
#include "common.cuh"

namespace ljmd {

template <int LANES>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int LANES>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int LANES, bool HALF, bool ENERGY>
__global__ void __launch_bounds__(256) k_force_mixed(const float4* __restrict__ hi, const float4* __restrict__ lo,
                                                     const uint32_t* __restrict__ row_ptr,
                                                     const uint32_t* __restrict__ col, int64_t N, Geom g,
                                                     LJConst c, float4* __restrict__ f, double* __restrict__ part) {
  const int lane = threadIdx.x & (LANES - 1);
  const int64_t gid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / LANES;
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / LANES;
  double pe_acc = 0.0, vir_acc = 0.0;
  for (int64_t i = gid; __any_sync(0xffffffffu, i < N); i += ngroups) {
    const bool valid = i < N;
    float fx = 0.f, fy = 0.f, fz = 0.f, pe = 0.f, vir = 0.f;
    if (valid) {
      const float4 hi_i = hi[i], lo_i = lo[i];
      const uint32_t b = row_ptr[i], e = row_ptr[i + 1];
      for (uint32_t k = b + lane; k < e; k += LANES) {
        const uint32_t j = col[k];
        const float4 hj = hi[j], lj = lo[j];
        float d[3];
        {
          const float dh0 = hj.x - hi_i.x, dh1 = hj.y - hi_i.y, dh2 = hj.z - hi_i.z;  // exact
          const float m0 = rintf(dh0 * g.inv_L), m1 = rintf(dh1 * g.inv_L), m2 = rintf(dh2 * g.inv_L);
          d[0] = fmaf(-m0, g.L_hi, dh0) + fmaf(-m0, g.L_lo, lj.x - lo_i.x);
          d[1] = fmaf(-m1, g.L_hi, dh1) + fmaf(-m1, g.L_lo, lj.y - lo_i.y);
          d[2] = fmaf(-m2, g.L_hi, dh2) + fmaf(-m2, g.L_lo, lj.z - lo_i.z);
        }
        const float r2 = fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2]));
        const float ri2 = __frcp_rn(r2);
        const float si = c.sig2f * ri2;
        const float s3i = si * si * si;
        const bool in = r2 < c.rc2f;
        float ff = fmaf(ri2 * s3i, fmaf(-c.f48, s3i, c.f24), c.f8c2);
        ff = in ? ff : 0.0f;
        fx = fmaf(ff, d[0], fx);
        fy = fmaf(ff, d[1], fy);
        fz = fmaf(ff, d[2], fz);
        if (HALF) atomicAdd(&f[j], make_float4(-ff * d[0], -ff * d[1], -ff * d[2], 0.0f));
        if (ENERGY) {
          const float v = c.e4 * fmaf(s3i, s3i - 1.0f, fmaf(c.c2f, r2, c.c0f));
          pe += in ? v : 0.0f;
          vir = fmaf(-ff, r2, vir);
        }
      }
    }
    fx = group_sum<LANES>(fx);
    fy = group_sum<LANES>(fy);
    fz = group_sum<LANES>(fz);
    if (valid && lane == 0) {
      if (HALF) atomicAdd(&f[i], make_float4(fx, fy, fz, 0.0f));
      else f[i] = make_float4(fx, fy, fz, 0.0f);
    }
    if (ENERGY) {
      pe_acc += (double)pe;
      vir_acc += (double)vir;
    }
  }
  if (ENERGY) {
    __shared__ double sh[32];
    const double tp = block_sum(pe_acc, sh);
    __syncthreads();
    const double tv = block_sum(vir_acc, sh);
    if (threadIdx.x == 0) {
      part[2 * (size_t)blockIdx.x] = tp;
      part[2 * (size_t)blockIdx.x + 1] = tv;
    }
  }
}

template <int LANES, bool HALF, bool ENERGY>
__global__ void __launch_bounds__(256) k_force_fp64(const dvec4* __restrict__ pos,
                                                    const uint32_t* __restrict__ row_ptr,
                                                    const uint32_t* __restrict__ col, int64_t N, Geom g, LJConst c,
                                                    dvec4* __restrict__ f, double* __restrict__ part) {
  const int lane = threadIdx.x & (LANES - 1);
  const int64_t gid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / LANES;
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / LANES;
  const double f24 = 24.0 * c.eps, f48 = 48.0 * c.eps, f8c2 = 8.0 * c.eps * c.c2 / c.sig2;
  const double e4 = 4.0 * c.eps, c2s = c.c2 / c.sig2;
  double pe_acc = 0.0, vir_acc = 0.0;
  for (int64_t i = gid; __any_sync(0xffffffffu, i < N); i += ngroups) {
    const bool valid = i < N;
    double fx = 0.0, fy = 0.0, fz = 0.0, pe = 0.0, vir = 0.0;
    if (valid) {
      const dvec4 qi = pos[i];
      const uint32_t b = row_ptr[i], e = row_ptr[i + 1];
      for (uint32_t k = b + lane; k < e; k += LANES) {
        const uint32_t j = col[k];
        const dvec4 qj = pos[j];
        double d0 = qj.x - qi.x, d1 = qj.y - qi.y, d2 = qj.z - qi.z;  // exact
        d0 = fma(-rint(d0 * g.inv_L64), g.L, d0);
        d1 = fma(-rint(d1 * g.inv_L64), g.L, d1);
        d2 = fma(-rint(d2 * g.inv_L64), g.L, d2);
        const double r2 = fma(d0, d0, fma(d1, d1, d2 * d2));
        const double ri2 = __drcp_rn(r2);
        const double si = c.sig2 * ri2;
        const double s3i = si * si * si;
        const bool in = r2 < c.rc2;
        double ff = fma(ri2 * s3i, fma(-f48, s3i, f24), f8c2);
        ff = in ? ff : 0.0;
        fx = fma(ff, d0, fx);
        fy = fma(ff, d1, fy);
        fz = fma(ff, d2, fz);
        if (HALF) {
          atomicAdd(&f[j].x, -ff * d0);
          atomicAdd(&f[j].y, -ff * d1);
          atomicAdd(&f[j].z, -ff * d2);
        }
        if (ENERGY) {
          const double v = e4 * fma(s3i, s3i - 1.0, fma(c2s, r2, c.c0));
          pe += in ? v : 0.0;
          vir = fma(-ff, r2, vir);
        }
      }
    }
    fx = group_sum<LANES>(fx);
    fy = group_sum<LANES>(fy);
    fz = group_sum<LANES>(fz);
    if (valid && lane == 0) {
      if (HALF) {
        atomicAdd(&f[i].x, fx);
        atomicAdd(&f[i].y, fy);
        atomicAdd(&f[i].z, fz);
      } else {
        f[i] = make_dvec4(fx, fy, fz, 0.0);
      }
    }
    if (ENERGY) {
      pe_acc += pe;
      vir_acc += vir;
    }
  }
  if (ENERGY) {
    __shared__ double sh[32];
    const double tp = block_sum(pe_acc, sh);
    __syncthreads();
    const double tv = block_sum(vir_acc, sh);
    if (threadIdx.x == 0) {
      part[2 * (size_t)blockIdx.x] = tp;
      part[2 * (size_t)blockIdx.x + 1] = tv;
    }
  }
}

template <int LANES, bool HALF, bool ENERGY>
static void launch_t(int precision, const void* pos, const float4* lo, const uint32_t* row_ptr, const uint32_t* col,
                     int64_t N, Geom g, LJConst c, void* f, double* part, int blocks, cudaStream_t s) {
  if (precision == LJ_MIXED)
    k_force_mixed<LANES, HALF, ENERGY><<<blocks, 256, 0, s>>>((const float4*)pos, lo, row_ptr, col, N, g, c,
                                                              (float4*)f, part);
  else
    k_force_fp64<LANES, HALF, ENERGY><<<blocks, 256, 0, s>>>((const dvec4*)pos, row_ptr, col, N, g, c,
                                                             (dvec4*)f, part);
}

template <int LANES>
static void launch_l(int precision, int half, int energy, const void* pos, const float4* lo,
                     const uint32_t* row_ptr, const uint32_t* col, int64_t N, Geom g, LJConst c, void* f,
                     double* part, int blocks, cudaStream_t s) {
  if (half) {
    if (energy) launch_t<LANES, true, true>(precision, pos, lo, row_ptr, col, N, g, c, f, part, blocks, s);
    else launch_t<LANES, true, false>(precision, pos, lo, row_ptr, col, N, g, c, f, part, blocks, s);
  } else {
    if (energy) launch_t<LANES, false, true>(precision, pos, lo, row_ptr, col, N, g, c, f, part, blocks, s);
    else launch_t<LANES, false, false>(precision, pos, lo, row_ptr, col, N, g, c, f, part, blocks, s);
  }
}

int launch_force(int precision, int half, int lanes, int energy, const void* pos, const float4* lo,
                 const uint32_t* row_ptr, const uint32_t* col, int64_t N, Geom g, LJConst c, void* f,
                 double* partials, cudaStream_t s) {
  // one group per key particle; grid capped so that per-block energy partials fit
  int64_t groups_per_block = 256 / lanes;
  int64_t b = (N + groups_per_block - 1) / groups_per_block;
  if (b < 1) b = 1;
  const int blocks = (int)(b < kMaxRedBlocks ? b : kMaxRedBlocks);
  switch (lanes) {
    case 1: launch_l<1>(precision, half, energy, pos, lo, row_ptr, col, N, g, c, f, partials, blocks, s); break;
    case 2: launch_l<2>(precision, half, energy, pos, lo, row_ptr, col, N, g, c, f, partials, blocks, s); break;
    case 4: launch_l<4>(precision, half, energy, pos, lo, row_ptr, col, N, g, c, f, partials, blocks, s); break;
    case 8: launch_l<8>(precision, half, energy, pos, lo, row_ptr, col, N, g, c, f, partials, blocks, s); break;
    case 16: launch_l<16>(precision, half, energy, pos, lo, row_ptr, col, N, g, c, f, partials, blocks, s); break;
    default: launch_l<32>(precision, half, energy, pos, lo, row_ptr, col, N, g, c, f, partials, blocks, s); break;
  }
  return blocks;
}

}  // namespace ljmd
