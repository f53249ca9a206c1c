// Pair-list construction (Alg. 1 over the cell grid of Sec. 2.2; the sorted list of Sec. 2.4).
//
// For each key particle i (cell order), the candidates are the particles of the cells adjacent
// to i's cell (27 for n >= 3 cells per side; all distinct cells for n < 3).  A candidate j is
// listed iff r_ij < r_s, where r_ij^2 = dx*dx + dy*dy + dz*dz is evaluated in FP64 without FMA
// on the fixed min-image differences, so the pair set equals an all-pairs brute force bit for bit.
//
// The FP64 test is only needed near r_s.  Each candidate is first tested in FP32 on the
// hi/lo split of the stored coordinates: the hi difference is exact (all hi parts are
// multiples of 2^(p-24) and |d| < 2^p), so d carries one FP32 rounding and r2f is within a
// few ulp of the exact r^2.  Outside the band [lo, hi) around r_s^2 (tens of ulp wide) the
// FP32 verdict equals the FP64 one; inside it the FP64 test decides.  This keeps the build on
// the FP32 pipe (FP64 runs at 1/64 of FP32 on this GPU).
//
// Two passes with identical candidate order: count (row sizes) and fill (SortedList).
#include "common.cuh"

namespace ljmd {

__device__ __forceinline__ bool pair_in_exact(const double* __restrict__ x, int64_t N, int64_t i, int64_t j,
                                              const Geom& g, double rs2) {
  double d[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double t = __dsub_rn(x[k * N + j], x[k * N + i]);  // exact difference of stored coordinates
    if (t > g.half_L) t = __dsub_rn(t, g.L);
    else if (t < -g.half_L) t = __dadd_rn(t, g.L);
    d[k] = t;
  }
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
  return r2 < rs2;
}

// FP32 squared distance from hi/lo parts with the periodic image chosen on the exact hi difference.
__device__ __forceinline__ float r2_hilo(const float4 hi_i, const float4 lo_i, const float4 hi_j, const float4 lo_j,
                                         const Geom& g) {
  float dh[3] = {hi_j.x - hi_i.x, hi_j.y - hi_i.y, hi_j.z - hi_i.z};
  float dl[3] = {lo_j.x - lo_i.x, lo_j.y - lo_i.y, lo_j.z - lo_i.z};
  float r2 = 0.0f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float m = rintf(dh[k] * g.inv_L);
    const float a = fmaf(-m, g.L_hi, dh[k]);  // exact
    const float b = fmaf(-m, g.L_lo, dl[k]);
    const float d = a + b;
    r2 = fmaf(d, d, r2);
  }
  return r2;
}

template <bool FILL>
__global__ void k_list(const float4* __restrict__ hi, const float4* __restrict__ lo, const double* __restrict__ x,
                       const uint32_t* __restrict__ cell_of, const uint32_t* __restrict__ cell_start, int64_t N,
                       Geom g, ListBand band, int half, uint32_t* __restrict__ row_count,
                       const uint32_t* __restrict__ row_ptr, uint32_t* __restrict__ col,
                       int32_t* __restrict__ status, unsigned long long* __restrict__ total64) {
  const int nn = g.n < 3 ? g.n : 3;  // distinct offsets per axis: {0}, {0,+1}, {0,+1,-1}
  const int offs[3] = {0, 1, -1};
  __shared__ unsigned long long blk_total;
  if (!FILL) {
    if (threadIdx.x == 0) blk_total = 0;
    __syncthreads();
  }
  unsigned long long my_total = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c = cell_of[i];
    const int cz = (int)(c % (uint32_t)g.n), cy = (int)((c / (uint32_t)g.n) % (uint32_t)g.n),
              cx = (int)(c / ((uint32_t)g.n * (uint32_t)g.n));
    const float4 hi_i = hi[i], lo_i = lo[i];
    uint32_t cnt = 0, pos = 0, end = 0;
    if (FILL) {
      pos = row_ptr[i];
      end = row_ptr[i + 1];
    }
    for (int a = 0; a < nn; ++a) {
      int ax = cx + offs[a];
      ax = ax < 0 ? ax + g.n : (ax >= g.n ? ax - g.n : ax);
      for (int b = 0; b < nn; ++b) {
        int by = cy + offs[b];
        by = by < 0 ? by + g.n : (by >= g.n ? by - g.n : by);
        for (int e = 0; e < nn; ++e) {
          int ez = cz + offs[e];
          ez = ez < 0 ? ez + g.n : (ez >= g.n ? ez - g.n : ez);
          const uint32_t cn = ((uint32_t)ax * (uint32_t)g.n + (uint32_t)by) * (uint32_t)g.n + (uint32_t)ez;
          const uint32_t jb = cell_start[cn], je = cell_start[cn + 1];
          for (uint32_t j = jb; j < je; ++j) {
            if ((int64_t)j == i || (half && (int64_t)j < i)) continue;
            const float r2f = r2_hilo(hi_i, lo_i, hi[j], lo[j], g);
            bool in = r2f < band.lo;
            if (!in && r2f < band.hi) in = pair_in_exact(x, N, i, j, g, band.rs2);
            if (in) {
              if (FILL) {
                if (pos < end) col[pos] = j;
                ++pos;
              } else {
                ++cnt;
              }
            }
          }
        }
      }
    }
    if (!FILL) {
      row_count[i] = cnt;
      my_total += cnt;
    } else if (pos != end) {
      atomicOr(status, LJ_ST_LIST_OVERFLOW);
    }
  }
  if (!FILL) {
    // 64-bit total of the row sizes (one global atomic per block): detects overflow of the
    // 32-bit row offsets
    atomicAdd(&blk_total, my_total);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(total64, blk_total);
  }
}

static int list_grid(int64_t N) {
  int64_t b = (N + 127) / 128;
  if (b < 1) b = 1;
  return (int)(b < 1048576 ? b : 1048576);
}

void launch_list_count(const void* hi, const float4* lo, const double* x, const uint32_t* cell_of,
                       const uint32_t* cell_start, int64_t N, Geom g, ListBand band, int half, int /*precision*/,
                       uint32_t* row_count, unsigned long long* total64, cudaStream_t s) {
  k_list<false><<<list_grid(N), 128, 0, s>>>((const float4*)hi, lo, x, cell_of, cell_start, N, g, band, half,
                                               row_count, nullptr, nullptr, nullptr, total64);
}

void launch_list_fill(const void* hi, const float4* lo, const double* x, const uint32_t* cell_of,
                      const uint32_t* cell_start, int64_t N, Geom g, ListBand band, int half, int /*precision*/,
                      const uint32_t* row_ptr, uint32_t* col, int32_t* status, cudaStream_t s) {
  k_list<true><<<list_grid(N), 128, 0, s>>>((const float4*)hi, lo, x, cell_of, cell_start, N, g, band, half,
                                              nullptr, row_ptr, col, status, nullptr);
}

}  // namespace ljmd
