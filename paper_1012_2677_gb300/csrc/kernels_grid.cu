// Cell grid (Sec. 2.2, Fig. 3): fold into the box, label by cell, count, scan, scatter;
// then reorder the particle arrays in cell order (Sec. 3.3).  Also the id-order copies.
#include "common.cuh"

namespace ljmd {

static int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (int)(b < 1048576 ? b : 1048576);
}

// Fold x_state into [offset, offset + L) (one correction per component, counted in img),
// label c = (cx n + cy) n + cz with cx = floor((x_state - offset) * n / L) clamped to [0, n-1],
// and count particles per cell.
// The lanes of a warp that land in one cell (neighbours in the previous cell order mostly do) add
// their count with one atomic.
__global__ void k_wrap_label(double* __restrict__ x, int32_t* __restrict__ img, int64_t N, Geom g,
                             uint32_t* __restrict__ cell_of, uint32_t* __restrict__ count,
                             int32_t* __restrict__ status) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const double top = g.offset + g.L;
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); i0 < N; i0 += stride) {
    const int64_t i = i0 + lane;
    uint32_t cell = 0xffffffffu;  // the warp's tail (no particle) takes part in the match only
    if (i < N) {
      int c[3];
      bool bad = false;
      for (int k = 0; k < 3; ++k) {
        double xs = x[k * N + i];
        if (!finite_d(xs)) bad = true;
        if (cmp_ge_d(xs, top)) {
          xs -= g.L;
          img[k * N + i] += 1;
          x[k * N + i] = xs;
        } else if (!cmp_ge_d(xs, g.offset)) {
          xs += g.L;
          img[k * N + i] -= 1;
          x[k * N + i] = xs;
        }
        const double rel = xs - g.offset;  // exact: both in [offset/2, 2 offset)
        int ck = floor_to_int(rel * g.inv_h);
        ck = ck < 0 ? 0 : (ck >= g.n ? g.n - 1 : ck);
        c[k] = ck;
      }
      if (bad) {
        atomicOr(status, LJ_ST_NONFINITE);
        c[0] = c[1] = c[2] = 0;
      }
      cell = ((uint32_t)c[0] * (uint32_t)g.n + (uint32_t)c[1]) * (uint32_t)g.n + (uint32_t)c[2];
      cell_of[i] = cell;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, cell);
    if (i < N && lane == __ffs(peers) - 1) atomicAdd(&count[cell], (uint32_t)__popc(peers));
  }
}

void launch_wrap_label(double* x, int32_t* img, int64_t N, Geom g, uint32_t* cell_of, uint32_t* cell_count,
                       int32_t* status, cudaStream_t s) {
  k_wrap_label<<<grid_for(N, 256), 256, 0, s>>>(x, img, N, g, cell_of, cell_count, status);
}

// ---------------------------------------------------------------------------------------------
// Exclusive scan, three passes: per-tile sums, scan of the tile sums (recursively), tile scan.
constexpr int kScanTile = 2048;  // 256 threads x 8 values

__global__ void k_tile_sums(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ sums, const int* __restrict__ pred) {
  if (pred && !*pred) return;  // predicated: skipped unless the flag is set
  __shared__ uint32_t sh[8];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t s = 0;
  for (int k = 0; k < 8; ++k) {
    const int64_t i = base + threadIdx.x + k * 256;
    if (i < n) s += in[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < 8; ++w) t += sh[w];
    sums[blockIdx.x] = t;
  }
}

// Scan of one tile: each thread owns 8 consecutive values; out[i] = base + exclusive prefix.
__global__ void k_tile_scan(const uint32_t* __restrict__ in, int64_t n, const uint32_t* __restrict__ tile_base,
                            uint32_t* __restrict__ out, const int* __restrict__ pred) {
  if (pred && !*pred) return;  // predicated: skipped unless the flag is set
  __shared__ uint32_t sh[8];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * 8;
  uint32_t v[8], t = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0u;
    t += v[k];
  }
  // inclusive warp scan of the per-thread totals
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t inc = t;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) sh[w] = inc;
  __syncthreads();
  uint32_t wbase = 0;
  for (int q = 0; q < w; ++q) wbase += sh[q];
  uint32_t run = (tile_base ? tile_base[blockIdx.x] : 0u) + wbase + inc - t;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 255) out[n] = run;  // total
}

size_t scan_tmp_words(int64_t n) {
  size_t words = 0;
  int64_t m = n;
  while (m > kScanTile) {
    const int64_t tiles = (m + kScanTile - 1) / kScanTile;
    words += 2 * (size_t)tiles + 1;
    m = tiles;
  }
  return words + 1;
}

int launch_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, cudaStream_t s, const int* pred) {
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles <= 1) {
    k_tile_scan<<<1, 256, 0, s>>>(in, n, nullptr, out, pred);
    return 1;
  }
  uint32_t* sums = tmp;                // [tiles]
  uint32_t* base = tmp + tiles;        // [tiles + 1]
  k_tile_sums<<<(int)tiles, 256, 0, s>>>(in, n, sums, pred);
  const int inner = launch_scan_u32(sums, base, tiles, tmp + 2 * tiles + 1, s, pred);
  k_tile_scan<<<(int)tiles, 256, 0, s>>>(in, n, base, out, pred);
  return inner + 2;
}

// ---------------------------------------------------------------------------------------------
// Scatter (Fig. 3 (ii)-(iii)): place each particle at its cell's pointer and advance it.
// The arrival order inside a cell is made deterministic afterwards by k_cell_rank (ids ascending).
// The lanes of a warp bound for one cell reserve their slots with one atomic.
__global__ void k_scatter(const uint32_t* __restrict__ cell_of, const uint32_t* __restrict__ start,
                          uint32_t* __restrict__ fill, uint32_t* __restrict__ perm, int64_t N, const int* __restrict__ pred) {
  if (pred && !*pred) return;  // predicated: skipped unless the flag is set
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); i0 < N; i0 += stride) {
    const int64_t i = i0 + lane;
    const uint32_t c = i < N ? cell_of[i] : 0xffffffffu;
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (lane == leader && i < N) base = atomicAdd(&fill[c], (uint32_t)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (i < N) perm[start[c] + base + (uint32_t)__popc(peers & ((1u << lane) - 1u))] = (uint32_t)i;
  }
}

void launch_scatter(const uint32_t* cell_of, const uint32_t* cell_start, uint32_t* cell_fill, uint32_t* perm,
                    int64_t N, cudaStream_t s, const int* pred) {
  k_scatter<<<grid_for(N, 256), 256, 0, s>>>(cell_of, cell_start, cell_fill, perm, N, pred);
}

// Inside each cell order the particles by id (the order of Fig. 3's counting sort, independent of the
// arrival order of the scatter's atomics): a group of 16 lanes per cell ranks each of the cell's
// entries of perm_in by the number of its entries with a smaller id and writes it at that rank of
// perm_out.
__global__ void k_cell_rank(const uint32_t* __restrict__ start, int64_t ncells, const uint32_t* __restrict__ perm_in,
                            const int32_t* __restrict__ id, uint32_t* __restrict__ perm_out,
                            const int* __restrict__ pred) {
  if (pred && !*pred) return;  // predicated: skipped unless the flag is set
  constexpr int G = 16;
  const int lane = threadIdx.x & (G - 1);
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
  // every lane of a warp runs the same number of iterations (its two groups' loops share the
  // shuffles), so the cell index steps by warps: c0 is the warp's first group
  const int64_t g0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
  for (int64_t c = g0; c - (g0 & 1) < ncells; c += groups) {
    const bool have = c < ncells;
    const uint32_t b = have ? start[c] : 0u;
    const int m = have ? (int)(start[c + 1] - b) : 0;
    const int mw = max(m, __shfl_xor_sync(0xffffffffu, m, G));  // the warp's larger cell
    for (int i0 = 0; i0 < mw; i0 += G) {
      const int i = i0 + lane;
      uint32_t p = 0;
      int key = 0x7fffffff;
      if (i < m) {
        p = perm_in[b + i];
        key = id[p];
      }
      int rank = 0;
      for (int j0 = 0; j0 < mw; j0 += G) {
        const int j = j0 + lane;
        const int other = j < m ? id[perm_in[b + j]] : 0x7fffffff;
        for (int t = 0; t < G; ++t) rank += __shfl_sync(0xffffffffu, other, t, G) < key ? 1 : 0;
      }
      if (i < m) perm_out[b + rank] = p;
    }
  }
}

void launch_cell_rank(const uint32_t* cell_start, int64_t ncells, const uint32_t* perm_in, const int32_t* id,
                      uint32_t* perm_out, cudaStream_t s, const int* pred) {
  int64_t b = (ncells + 15) / 16;  // 16 cells per 256-thread block
  if (b < 1) b = 1;
  if (b > 1048576) b = 1048576;
  k_cell_rank<<<(int)b, 256, 0, s>>>(cell_start, ncells, perm_in, id, perm_out, pred);
}

// ---------------------------------------------------------------------------------------------
// Gathers: out[k] = in[perm[k]].

// The particle state in one pass (perm read once): positions and velocities (FP64 x 3), ids,
// image counts (3) and, FB = 16 or 32, the last forces (float4 or double4 records).
template <int FB>
__global__ void k_gather_state(const uint32_t* __restrict__ perm, int64_t N, const double* __restrict__ x,
                               double* __restrict__ x2, const double* __restrict__ v, double* __restrict__ v2,
                               const int32_t* __restrict__ id, int32_t* __restrict__ id2,
                               const int32_t* __restrict__ img, int32_t* __restrict__ img2,
                               const uint4* __restrict__ f, uint4* __restrict__ f2, const int* __restrict__ pred) {
  if (pred && !*pred) return;  // predicated: skipped unless the flag is set
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    const size_t p = perm[k];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x2[c * N + k] = x[c * N + p];
      v2[c * N + k] = v[c * N + p];
      img2[c * N + k] = img[c * N + p];
    }
    id2[k] = id[p];
    if (FB == 16) f2[k] = f[p];
    if (FB == 32) {
      f2[2 * k] = f[2 * p];
      f2[2 * k + 1] = f[2 * p + 1];
    }
  }
}
void launch_gather_state(const uint32_t* perm, int64_t N, const double* x, double* x2, const double* v, double* v2,
                         const int32_t* id, int32_t* id2, const int32_t* img, int32_t* img2, const void* f, void* f2,
                         int fbytes, cudaStream_t s, const int* pred) {
  const uint4* fi = (const uint4*)f;
  uint4* fo = (uint4*)f2;
  if (fbytes == 16)
    k_gather_state<16><<<grid_for(N, 256), 256, 0, s>>>(perm, N, x, x2, v, v2, id, id2, img, img2, fi, fo, pred);
  else if (fbytes == 32)
    k_gather_state<32><<<grid_for(N, 256), 256, 0, s>>>(perm, N, x, x2, v, v2, id, id2, img, img2, fi, fo, pred);
  else
    k_gather_state<0><<<grid_for(N, 256), 256, 0, s>>>(perm, N, x, x2, v, v2, id, id2, img, img2, fi, fo, pred);
}
// ---------------------------------------------------------------------------------------------
// Copies between the sorted SoA state and caller-order AoS (x[3 id + k]).
__global__ void k_scatter_back_f64x3(const double* __restrict__ in, double* __restrict__ out,
                                     const int32_t* __restrict__ id, int64_t N, double sub) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = id[k];
    out[3 * p + 0] = in[k] - sub;
    out[3 * p + 1] = in[N + k] - sub;
    out[3 * p + 2] = in[2 * N + k] - sub;
  }
}
void launch_scatter_back_f64x3(const double* in, double* out_idorder, const int32_t* id, int64_t N, double sub,
                               cudaStream_t s) {
  k_scatter_back_f64x3<<<grid_for(N, 256), 256, 0, s>>>(in, out_idorder, id, N, sub);
}

__global__ void k_scatter_back_f32x4(const float4* __restrict__ in, double* __restrict__ out,
                                     const int32_t* __restrict__ id, int64_t N) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = id[k];
    const float4 f = in[k];
    out[3 * p + 0] = f.x;
    out[3 * p + 1] = f.y;
    out[3 * p + 2] = f.z;
  }
}
void launch_scatter_back_f32x4_to_f64x3(const float4* in, double* out, const int32_t* id, int64_t N,
                                        cudaStream_t s) {
  k_scatter_back_f32x4<<<grid_for(N, 256), 256, 0, s>>>(in, out, id, N);
}

__global__ void k_scatter_back_f64x4(const dvec4* __restrict__ in, double* __restrict__ out,
                                     const int32_t* __restrict__ id, int64_t N) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = id[k];
    const dvec4 f = in[k];
    out[3 * p + 0] = f.x;
    out[3 * p + 1] = f.y;
    out[3 * p + 2] = f.z;
  }
}
void launch_scatter_back_f64x4_to_f64x3(const dvec4* in, double* out, const int32_t* id, int64_t N,
                                        cudaStream_t s) {
  k_scatter_back_f64x4<<<grid_for(N, 256), 256, 0, s>>>(in, out, id, N);
}

__global__ void k_scatter_back_i32x3(const int32_t* __restrict__ in, int32_t* __restrict__ out,
                                     const int32_t* __restrict__ id, int64_t N) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = id[k];
    out[3 * p + 0] = in[k];
    out[3 * p + 1] = in[N + k];
    out[3 * p + 2] = in[2 * N + k];
  }
}
void launch_scatter_back_i32x3(const int32_t* in, int32_t* out, const int32_t* id, int64_t N, cudaStream_t s) {
  k_scatter_back_i32x3<<<grid_for(N, 256), 256, 0, s>>>(in, out, id, N);
}

// Caller-order AoS (x[3 p + k], v or NULL) into the SoA state; id = p.  Positions are folded
// into [0, L) (img counts the folds, so x_in = x + img L) and stored as offset + x.
__global__ void k_load_state(const double* __restrict__ xin, const double* __restrict__ vin, double* __restrict__ x,
                             double* __restrict__ v, int32_t* __restrict__ id, int32_t* __restrict__ img, int64_t N,
                             double offset, double L) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    for (int k = 0; k < 3; ++k) {
      const double xi = xin[3 * p + k];
      double m = floor(xi / L);
      double xr = xi - m * L;
      if (xr >= L) {
        xr -= L;
        m += 1.0;
      } else if (xr < 0.0) {
        xr += L;
        m -= 1.0;
      }
      x[k * N + p] = offset + xr;
      v[k * N + p] = vin ? vin[3 * p + k] : 0.0;
      img[k * N + p] = (int32_t)m;
    }
    id[p] = (int32_t)p;
  }
}
void launch_load_state(const double* x_in, const double* v_in, double* x, double* v, int32_t* id, int32_t* img,
                       int64_t N, double offset, double L, cudaStream_t s) {
  k_load_state<<<grid_for(N, 256), 256, 0, s>>>(x_in, v_in, x, v, id, img, N, offset, L);
}

__global__ void k_iota(int32_t* __restrict__ id, int64_t N) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x)
    id[p] = (int32_t)p;
}
void launch_iota_i32(int32_t* id, int64_t N, cudaStream_t s) { k_iota<<<grid_for(N, 256), 256, 0, s>>>(id, N); }

}  // namespace ljmd
