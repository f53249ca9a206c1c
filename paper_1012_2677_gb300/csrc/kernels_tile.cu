// Cell-column tiles staged in shared memory: pair-list construction (Alg. 1 over the grid of
// Sec. 2.2, stored as the sorted list of Sec. 2.4) and the force over that list (Alg. 4-6).
//
// A tile is T consecutive cells along z of one (cx, cy) column.  Its CTA stages the particles
// of the 9 neighbouring columns over the cells z0-1 .. z0+T (9 (T+2) cells, wrapped
// periodically) into shared memory.  The cells of one column are contiguous in the cell-sorted
// particle arrays (except where z wraps), so each column is one to three contiguous ranges:
// one lane per column issues asynchronous bulk copies (cp.async.bulk) of those ranges, plus
// the tile's rows and its list segment, all completing on one mbarrier that the CTA waits on
// (bounded).  The periodic image shifts (-L, 0, +L per axis) are then added in shared memory.
//
// Mixed form, force and adjoint kernels: the copies are the fixed-point coordinates of the stored
// FP64 positions (X = round(x / u) mod 2^32, u = 2^-qk, one 16-byte record per particle with the
// sorted index in w), the image shift is the integer round(L / u), and a partner difference is
// the exact integer X_j - X_i converted once to FP32.  List kernels: the FP32 hi parts (top 24
// significand bits) of the stored coordinates, whose differences are exact.  FP64 form: the FP64
// coordinates, the periodic images put in place when staged (one rounding per staged coordinate).
//
// The list holds 16-bit indices into the key particle's staged tile; rows are (start, length)
// per particle; the rows of one tile form one contiguous segment, padded to 8 entries so that
// it can be bulk-copied.  If the box has fewer than 3 cells per side the whole box is one tile
// (all particles staged directly, no shifts, image chosen per pair).
//
// List construction: one lane per key particle tests the three cells around its own in each of
// the 9 neighbour columns (the 27 cells of Alg. 1) from shared memory, FP32 on hi differences,
// which are exact, so r^2 is within a bounded error of the FP64 value; inside that band the FP64
// no-FMA test of the oracle decides, and the pair set equals brute force bit for bit.  The kept
// bits are counted, one atomic per tile reserves the tile's segment, and the entries are written
// from the bits (k_list_win).  The whole-box case (k_list_tile) takes a warp per key particle
// with ballot compaction.
#include "common.cuh"

#include <type_traits>

namespace ljmd {

constexpr int kTileThreads = 256;
constexpr int kWarps = kTileThreads / 32;
constexpr int kMaxCells = 9 * (kMaxTileT + 2);

// Budget of the waits for a tile's copies and for the other warps of the pipelined kernel (SM
// clock cycles); the waits that let copies in flight land before a CTA leaves keep kWaitBudget.
// Lowered only by ljmd_set_wait_budget, to drive the timeout paths in tests.
__device__ long long g_wait_budget = kWaitBudget;
__device__ __forceinline__ long long wait_budget() { return g_wait_budget; }

struct TileInfo {
  int cx, cy, z0, Tp;
};

__device__ __forceinline__ TileInfo tile_info(int64_t t64, const TileArgs& ta) {
  TileInfo ti;
  const unsigned t = (unsigned)t64;  // tiles < 2^31 (n <= 1024)
  const unsigned tz = t % (unsigned)ta.ntz;
  const unsigned r = t / (unsigned)ta.ntz;
  ti.cy = (int)(r % (unsigned)ta.n);
  ti.cx = (int)(r / (unsigned)ta.n);
  ti.z0 = (int)tz * ta.T;
  ti.Tp = min(ta.T, ta.n - ti.z0);
  return ti;
}

// Shared bookkeeping of one staged tile.
struct TileShared {
  int offq[kMaxCells + 1];  // staged index of the first particle of cell q = k (Tp+2) + m
  int g0[kMaxCells];        // sorted (global) index of the first particle of cell q
  int ncol, ncell, total;   // cells per column, staged cells, staged particles
  int own0, own1;           // staged range of the tile's own particles
  int gown0;                // sorted index of the first own particle
  unsigned list_base, list_len;  // the tile's (padded) list segment
  int row_off;              // index of the first own row in the staged row copy
};

// Wrapped coordinate and image shift (-1, 0, +1) of a neighbour cell index.
__device__ __forceinline__ int wrap_cell(int c, int n, int& shift) {
  shift = 0;
  if (c < 0) {
    c += n;
    shift = -1;
  } else if (c >= n) {
    c -= n;
    shift = 1;
  }
  return c;
}

__device__ __forceinline__ uint32_t cell_of_q(const TileInfo& ti, int n, int ncol, int q, int& sx, int& sy, int& sz) {
  const int k = q / ncol, m = q - (q / ncol) * ncol;
  const int X = wrap_cell(ti.cx + k / 3 - 1, n, sx);
  const int Y = wrap_cell(ti.cy + k % 3 - 1, n, sy);
  const int Z = wrap_cell(ti.z0 - 1 + m, n, sz);
  return ((uint32_t)X * (uint32_t)n + (uint32_t)Y) * (uint32_t)n + (uint32_t)Z;
}

// Cell bounds of the tile's 9 (Tp + 2) staged cells and their prefix (one warp).  Returns false
// (all threads) if the tile exceeds the staged capacity.
__device__ __forceinline__ bool stage_offsets(const TileInfo& ti, const TileArgs& ta, const uint32_t* __restrict__ cs,
                                              TileShared& S) {
  const int ncol = ti.Tp + 2;
  const int ncell = 9 * ncol;
  for (int q = threadIdx.x; q < ncell; q += blockDim.x) {
    int sx, sy, sz;
    const uint32_t c = cell_of_q(ti, ta.n, ncol, q, sx, sy, sz);
    const uint32_t a = cs[c], b = cs[c + 1];
    S.g0[q] = (int)a;
    S.offq[q + 1] = (int)(b - a);
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int run = 0;
    for (int base = 0; base < ncell; base += 32) {
      const int q = base + lane;
      const int v = q < ncell ? S.offq[q + 1] : 0;
      int inc = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      if (q < ncell) S.offq[q + 1] = run + inc;
      run += __shfl_sync(0xffffffffu, inc, 31);
    }
    __syncwarp();
    if (lane == 0) {
      S.offq[0] = 0;
      S.ncol = ncol;
      S.ncell = ncell;
      S.total = run;
      S.own0 = S.offq[4 * ncol + 1];
      S.own1 = S.offq[4 * ncol + ti.Tp + 1];
      S.gown0 = S.g0[4 * ncol + 1];
    }
  }
  __syncthreads();
  return S.total <= ta.max_staged;
}

// Cell bounds of a tile's staged cells held in one warp's registers (lane l: cells l, l + 32, ...),
// loaded a tile ahead of their use so the bookkeeping never waits on memory.
constexpr int kPfRounds = (kMaxCells + 31) / 32;
struct TilePrefetch {
  TileInfo ti;
  uint2 tl;
  uint32_t a[kPfRounds], b[kPfRounds];
};

__device__ __forceinline__ void tile_prefetch(int64_t t, const TileArgs& ta, const uint32_t* __restrict__ cs,
                                              const uint2* __restrict__ tile_list, TilePrefetch& pf, int lane) {
  pf.ti = tile_info(t, ta);
  const int ncol = pf.ti.Tp + 2, ncell = 9 * ncol;
  pf.tl = tile_list ? tile_list[t] : make_uint2(0u, 0u);
#pragma unroll
  for (int r = 0; r < kPfRounds; ++r) {
    const int q = 32 * r + lane;
    pf.a[r] = pf.b[r] = 0u;
    if (q < ncell) {
      int sx, sy, sz;
      const uint32_t c = cell_of_q(pf.ti, ta.n, ncol, q, sx, sy, sz);
      pf.a[r] = cs[c];
      pf.b[r] = cs[c + 1];
    }
  }
}

// The bookkeeping of stage_offsets done by one warp from prefetched bounds (no CTA barrier, the
// other warps keep computing); also the tile's list segment.
__device__ __forceinline__ bool tile_prepare_pf(const TilePrefetch& pf, const TileArgs& ta, TileShared& S, int lane) {
  const int ncol = pf.ti.Tp + 2, ncell = 9 * ncol;
  int run = 0;
#pragma unroll
  for (int r = 0; r < kPfRounds; ++r) {
    if (32 * r >= ncell) break;
    const int q = 32 * r + lane;
    int inc = q < ncell ? (int)(pf.b[r] - pf.a[r]) : 0;
    if (q < ncell) S.g0[q] = (int)pf.a[r];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (q < ncell) S.offq[q + 1] = run + inc;
    run += __shfl_sync(0xffffffffu, inc, 31);
  }
  __syncwarp();
  if (lane == 0) {
    S.offq[0] = 0;
    S.ncol = ncol;
    S.ncell = ncell;
    S.total = run;
    S.own0 = S.offq[4 * ncol + 1];
    S.own1 = S.offq[4 * ncol + pf.ti.Tp + 1];
    S.gown0 = S.g0[4 * ncol + 1];
    S.list_base = pf.tl.x;
    S.list_len = pf.tl.y;
  }
  __syncwarp();
  return run <= ta.max_staged;
}

// Cell bounds of a tile's staged cells copied asynchronously into shared memory (one warp; lane m
// takes cell m of every column).  Nothing waits for the loads until tile_prepare_async.
__device__ __forceinline__ void tile_prefetch_async(const TileInfo& ti, const TileArgs& ta,
                                                    const uint32_t* __restrict__ cs, uint32_t* pa, uint32_t* pb,
                                                    int lane) {
  const int ncol = ti.Tp + 2;
  if (lane >= ncol) return;
  int sz;
  const uint32_t Z = (uint32_t)wrap_cell(ti.z0 - 1 + lane, ta.n, sz);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    int sx, sy;
    const uint32_t X = (uint32_t)wrap_cell(ti.cx + k / 3 - 1, ta.n, sx);
    const uint32_t Y = (uint32_t)wrap_cell(ti.cy + k % 3 - 1, ta.n, sy);
    const uint32_t c = (X * (uint32_t)ta.n + Y) * (uint32_t)ta.n + Z;
    cp_async4(pa + k * ncol + lane, cs + c);
    cp_async4(pb + k * ncol + lane, cs + c + 1);
  }
}

// The bookkeeping of stage_offsets done by one warp from the bounds of tile_prefetch_async.
__device__ __forceinline__ bool tile_prepare_async(const TileInfo& ti, const uint32_t* pa, const uint32_t* pb,
                                                   const TileArgs& ta, TileShared& S, int lane) {
  cp_async_wait_all();
  __syncwarp();
  const int ncol = ti.Tp + 2, ncell = 9 * ncol;
  int run = 0;
  for (int base = 0; base < ncell; base += 32) {
    const int q = base + lane;
    int inc = 0;
    if (q < ncell) {
      const uint32_t a = pa[q];
      inc = (int)(pb[q] - a);
      S.g0[q] = (int)a;
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (q < ncell) S.offq[q + 1] = run + inc;
    run += __shfl_sync(0xffffffffu, inc, 31);
  }
  __syncwarp();  // the bounds are read before the next prefetch overwrites them
  if (lane == 0) {
    S.offq[0] = 0;
    S.ncol = ncol;
    S.ncell = ncell;
    S.total = run;
    S.own0 = S.offq[4 * ncol + 1];
    S.own1 = S.offq[4 * ncol + ti.Tp + 1];
    S.gown0 = S.g0[4 * ncol + 1];
    S.list_base = 0;
    S.list_len = 0;
  }
  __syncwarp();
  return run <= ta.max_staged;
}

// Staged cell of staged slot s: the largest q with offq[q] <= s.
__device__ __forceinline__ int slot_cell(const TileShared& S, int s) {
  int lo = 0, hi = S.ncell - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (S.offq[mid] <= s) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Shared-memory layout of a staged tile (byte offsets from the dynamic shared base).
struct TileLayout {
  size_t pos;    // MIXED: fixed-point uint4 [ms] (force, adjoint) or hi float4 [ms] (list); FP64: dvec4 [ms]
  size_t gid;    // int [ms] (where the sorted index is not carried in the staged record)
  size_t rows;   // uint2 [max_own + 2] (force only)
  size_t ent;    // uint16 [list_cap] (force only)
  size_t cnt;    // int [max_own] (list only), then pre [max_own], then masks [max_own * max_chunks]
  size_t total;
};

static __host__ __device__ __forceinline__ size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

__host__ __device__ __forceinline__ TileLayout tile_layout(const TileArgs& ta, bool mixed, bool force,
                                                           bool gid = true) {
  TileLayout L;
  const size_t ms = (size_t)ta.max_staged;
  L.pos = 0;
  size_t o = align16(ms * (mixed ? 16 : 32));
  L.gid = o;
  if (gid) o += align16(ms * 4);  // the full-list force kernel needs no sorted indices
  L.rows = o;
  L.ent = o;
  L.cnt = o;
  if (force) {
    o += align16(8 * ((size_t)ta.max_own + 2));
    L.ent = o;
    if (!ta.whole) o += align16(2 * (size_t)ta.list_cap);
  } else {
    o += align16(8 * (size_t)ta.max_own + 4 * (size_t)ta.max_own * ta.max_chunks);
  }
  L.total = o;
  return L;
}

// Issue the bulk copies of one tile (warp `issuer`; lane k < 9 handles column k, lane 9 the rows
// and list segment), all completing on `bar`.  Copies: positions (fixed-point records, hi or FP64), and for the
// force kernel the own rows and the list segment.  No barrier inside: the other warps go on.
template <bool MIXED, bool FORCE>
__device__ __forceinline__ void stage_issue(const TileInfo& ti, const TileArgs& ta, const void* __restrict__ pos,
                                            const uint2* __restrict__ rows, const uint16_t* __restrict__ ent,
                                            TileShared& S, unsigned char* smem, const TileLayout& L, uint64_t* bar,
                                            int issuer = 0) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned bpp = MIXED ? 16u : 32u;
  if (warp != issuer) return;
  unsigned bytes = (unsigned)S.total * bpp;
  int r0 = 0, r1 = 0;
  const int n_own = S.own1 - S.own0;
  if (FORCE) {
    r0 = S.gown0 & ~1;
    r1 = (S.gown0 + n_own + 1) & ~1;
    if (n_own > 0) bytes += 8u * (unsigned)(r1 - r0);
    if (S.list_len <= (unsigned)ta.list_cap) bytes += 2u * S.list_len;
  }
  if (lane == 0) {
    fence_proxy_async_smem();
    mbar_arrive_expect(bar, bytes);
  }
  __syncwarp();
  if (lane < 9) {
    // column `lane`: cells z0-1 .. z0+Tp wrapped in z; they are contiguous in the sorted arrays
    // except where z wraps (first cell when z0 = 0, last cell when z0 + Tp = n), so one to two runs
    const int k = lane, ncol = S.ncol;
    int cut0 = 0, cut1 = ncol;  // middle run [cut0, cut1); wrapped single cells outside it
    if (ti.z0 == 0) cut0 = 1;
    if (ti.z0 + ti.Tp == ta.n) cut1 = ncol - 1;
    const int bounds[4] = {0, cut0, cut1, ncol};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int m0 = bounds[r], m1 = bounds[r + 1];
      if (m1 <= m0) continue;
      const int q0 = k * ncol + m0;
      const unsigned n = (unsigned)(S.offq[k * ncol + m1] - S.offq[q0]);
      if (n > 0) {
        const size_t gsrc = (size_t)S.g0[q0];
        const size_t dst = (size_t)S.offq[q0];
        if (MIXED) {
          bulk_g2s(smem + L.pos + 16 * dst, (const uint4*)pos + gsrc, 16u * n, bar);
        } else {
          bulk_g2s(smem + L.pos + 32 * dst, (const dvec4*)pos + gsrc, 32u * n, bar);
        }
      }
    }
  } else if (FORCE && lane == 9) {
    if (n_own > 0) bulk_g2s(smem + L.rows, rows + r0, 8u * (unsigned)(r1 - r0), bar);
    if (S.list_len > 0 && S.list_len <= (unsigned)ta.list_cap)
      bulk_g2s(smem + L.ent, ent + S.list_base, 2u * S.list_len, bar);
    S.row_off = S.gown0 - r0;
  }
}

// Image shift of one staged fixed-point coordinate by s L (s = -1, 0, +1): the integer s round(L / u)
// added modulo 2^32 (exact; the image carries the rounding of L / u, at most u / 2).
__device__ __forceinline__ uint32_t shift_q(uint32_t q, int s, const Geom& g) {
  return s > 0 ? q + g.Lq : (s < 0 ? q - g.Lq : q);
}

// Wait (all threads, bounded) for the copies of a staged tile, then fill in the image shifts
// (mixed: added to the fixed-point record or to hi; FP64: s L added to the coordinates) and, if
// wanted, the sorted indices.  Returns false
// (all threads) on timeout, after recording it; the caller drains any other copies in flight.
template <bool MIXED, bool FORCE>
__device__ __forceinline__ bool stage_finish(const TileInfo& ti, const TileArgs& ta, const Geom& g, TileShared& S,
                                             unsigned char* smem, const TileLayout& L, uint64_t* bar,
                                             uint32_t& phase, bool want_gid, int32_t* status) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // one thread polls the barrier; the others wait at the CTA barrier without taking issue slots
  bool ok = true;
  if (threadIdx.x == 0) ok = mbar_wait(bar, phase, wait_budget());
  ok = __syncthreads_and(ok) != 0;
  if (!ok) {
    if (threadIdx.x == 0) {
      atomicOr(status, LJ_ST_TIMEOUT);
      mbar_wait(bar, phase, kWaitBudget);  // let copies in flight land before the CTA leaves
    }
    __syncthreads();
    return false;
  }
  phase ^= 1u;
  // interior tiles (no periodic image among the staged cells) need no shifts
  const bool interior = ti.cx >= 1 && ti.cx <= ta.n - 2 && ti.cy >= 1 && ti.cy <= ta.n - 2 && ti.z0 >= 1 &&
                        ti.z0 + ti.Tp <= ta.n - 1;
  if (interior && !want_gid) return true;
  for (int q = warp; q < S.ncell; q += (int)(blockDim.x >> 5)) {
    int sx = 0, sy = 0, sz = 0;
    if (!interior) cell_of_q(ti, ta.n, S.ncol, q, sx, sy, sz);
    const bool shifted = (sx | sy | sz) != 0;
    if (!shifted && !want_gid) continue;
    const int a = S.offq[q], b = S.offq[q + 1], gq = S.g0[q];
    for (int s = a + lane; s < b; s += 32) {
      if (MIXED) {
        if (shifted) {
          if (FORCE) {
            uint4* q = (uint4*)(smem + L.pos) + s;
            q->x = shift_q(q->x, sx, g);
            q->y = shift_q(q->y, sy, g);
            q->z = shift_q(q->z, sz, g);
          } else {  // list filter: hi only; a rounding of hi stays inside the FP32 band
            float4* h = (float4*)(smem + L.pos) + s;
            h->x = fmaf((float)sx, g.L_hi, h->x);
            h->y = fmaf((float)sy, g.L_hi, h->y);
            h->z = fmaf((float)sz, g.L_hi, h->z);
          }
        }
      } else if (shifted) {  // the image itself: one rounding per staged coordinate, none per pair
        dvec4* p = (dvec4*)(smem + L.pos) + s;
        p->x += (double)sx * g.L;
        p->y += (double)sy * g.L;
        p->z += (double)sz * g.L;
      }
      if (want_gid) ((int*)(smem + L.gid))[s] = gq + (s - a);
    }
  }
  // these generic writes precede later bulk copies into the same bytes
  fence_proxy_async_smem();
  __syncthreads();
  return true;
}

// Issue, wait and fix up one tile (single-buffered use).
template <bool MIXED, bool FORCE>
__device__ __forceinline__ bool stage_copy_async(const TileInfo& ti, const TileArgs& ta, const Geom& g,
                                                 const void* __restrict__ pos, const uint2* __restrict__ rows,
                                                 const uint16_t* __restrict__ ent, TileShared& S, unsigned char* smem,
                                                 const TileLayout& L, uint64_t* bar, uint32_t& phase, bool want_gid,
                                                 int32_t* status) {
  stage_issue<MIXED, FORCE>(ti, ta, pos, rows, ent, S, smem, L, bar);
  return stage_finish<MIXED, FORCE>(ti, ta, g, S, smem, L, bar, phase, want_gid, status);
}

// Whole box as one tile (fewer than 3 cells per side): everything staged directly, no shifts.
// GID: also the sorted indices (every layout but the mixed force and adjoint kernels', whose
// fixed-point records carry them).
template <bool MIXED, bool GID>
__device__ __forceinline__ void stage_whole(int64_t N, const void* __restrict__ pos, TileShared& S,
                                            unsigned char* smem, const TileLayout& L) {
  for (int e = threadIdx.x; e < N; e += blockDim.x) {
    if (MIXED) {
      ((uint4*)(smem + L.pos))[e] = ((const uint4*)pos)[e];
    } else {
      dvec4 p = ((const dvec4*)pos)[e];
      p.w = 13.0;  // no shift
      ((dvec4*)(smem + L.pos))[e] = p;
    }
    if (GID) ((int*)(smem + L.gid))[e] = e;
  }
  if (threadIdx.x == 0) {
    S.ncol = 1;
    S.ncell = 1;
    S.total = (int)N;
    S.own0 = 0;
    S.own1 = (int)N;
    S.gown0 = 0;
    S.offq[0] = 0;
    S.offq[1] = (int)N;
  }
}

// Exact list test of the oracle (FP64, fixed min-image formula, no FMA) on stored coordinates.
__device__ __forceinline__ bool pair_in_exact(const double* __restrict__ x, int64_t N, int i, int j, const Geom& g,
                                              double rs2) {
  double d[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double t = __dsub_rn(x[k * N + j], x[k * N + i]);
    if (t > g.half_L) t = __dsub_rn(t, g.L);
    else if (t < -g.half_L) t = __dadd_rn(t, g.L);
    d[k] = t;
  }
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
  return r2 < rs2;
}

// Candidate test in FP32 on staged copies (exact hi differences for the mixed form; the FP64
// form rounds its exact difference), then the exact FP64 test inside the band.
template <bool MIXED, bool WHOLE>
__device__ __forceinline__ bool candidate_in(const unsigned char* smem, const TileLayout& L, int li, int lj,
                                             const double* __restrict__ x, int64_t N, const Geom& g,
                                             const ListBand& band) {
  float r2;
  if (MIXED) {
    const float4 a = ((const float4*)(smem + L.pos))[li], b = ((const float4*)(smem + L.pos))[lj];
    float dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;  // exact
    if (WHOLE) {
      dx = fmaf(-rintf(dx * g.inv_L), g.L_hi, dx);
      dy = fmaf(-rintf(dy * g.inv_L), g.L_hi, dy);
      dz = fmaf(-rintf(dz * g.inv_L), g.L_hi, dz);
    }
    r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  } else {
    const dvec4 a = ((const dvec4*)(smem + L.pos))[li], b = ((const dvec4*)(smem + L.pos))[lj];
    double dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;  // staged tiles: images already in place
    if (WHOLE) {
      dx = fma(-rint(dx * g.inv_L64), g.L, dx);
      dy = fma(-rint(dy * g.inv_L64), g.L, dy);
      dz = fma(-rint(dz * g.inv_L64), g.L, dz);
    }
    const float fx = (float)dx, fy = (float)dy, fz = (float)dz;
    r2 = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
  }
  if (r2 < band.lo) return true;
  if (r2 >= band.hi) return false;
  const int* gid = (const int*)(smem + L.gid);
  return pair_in_exact(x, N, gid[li], gid[lj], g, band.rs2);
}

__device__ __forceinline__ int own_cell(const TileShared& S, int l, int Tp) {
  const int base = 4 * S.ncol;
  int m = 1;
  while (m < Tp && l >= S.offq[base + m + 1]) ++m;
  return m;
}

// ---------------------------------------------------------------------------------------------
// Batched replicas: the tile geometry of a replica (capacities stay the batch's).
__device__ __forceinline__ void replica_view(const ReplicaGeo& rg, TileArgs& ta, Geom& g) {
  ta.n = rg.n;
  ta.T = rg.T;
  ta.ntz = rg.ntz;
  ta.whole = 0;
  ta.ntiles = (int64_t)rg.n * rg.n * rg.ntz;
  g = rg.g;
}

template <bool MIXED, bool HALF, bool WHOLE>
__global__ void __launch_bounds__(kTileThreads, 4)
    k_list_tile(const void* __restrict__ pos, const double* __restrict__ x, const uint32_t* __restrict__ cs, int64_t N,
                Geom g, TileArgs ta, ListBand band, uint2* __restrict__ rows, uint2* __restrict__ tile_list,
                uint16_t* __restrict__ ent, uint64_t cap, unsigned long long* __restrict__ counter,
                unsigned int* __restrict__ max_list, int32_t* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ TileShared S;
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_ok;
  __shared__ unsigned int s_base;
  const TileLayout L = tile_layout(ta, MIXED, false);
  int* sh_gid = (int*)(smem + L.gid);
  int* s_cnt = (int*)(smem + L.cnt);                  // [max_own]
  int* s_pre = s_cnt + ta.max_own;                    // [max_own]
  uint32_t* masks = (uint32_t*)(s_pre + ta.max_own);  // [max_own * max_chunks]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  uint32_t phase = 0;
  if (!WHOLE) {
    if (threadIdx.x == 0) {
      mbar_init(&bar, 1);
      fence_proxy_async_smem();
    }
    __syncthreads();
  }

  for (int64_t t = blockIdx.x; t < ta.ntiles; t += gridDim.x) {
    TileInfo ti{0, 0, 0, 1};
    if (WHOLE) {
      stage_whole<MIXED, true>(N, pos, S, smem, L);
    } else {
      ti = tile_info(t, ta);
      if (!stage_offsets(ti, ta, cs, S)) {
        if (threadIdx.x == 0) atomicOr(status, LJ_ST_CELL_RANGE);
        __syncthreads();
        continue;
      }
      if (!stage_copy_async<MIXED, false>(ti, ta, g, pos, nullptr, nullptr, S, smem, L, &bar, phase, true, status))
        return;
    }
    __syncthreads();
    const int n_own = S.own1 - S.own0;
    const int nk = WHOLE ? 1 : 9;
    if (n_own > ta.max_own) {  // sizing inconsistency: record and skip the tile
      if (threadIdx.x == 0) atomicOr(status, LJ_ST_CELL_RANGE);
      __syncthreads();
      continue;
    }
    // phase 1: test, keep ballots, count
    for (int o = warp; o < n_own; o += kWarps) {
      const int l = S.own0 + o;
      const int gi = sh_gid[l];
      const int m = WHOLE ? 0 : own_cell(S, l, ti.Tp);
      int cnt = 0, c = 0;
      for (int k = 0; k < nk; ++k) {
        const int a = WHOLE ? 0 : S.offq[k * S.ncol + m - 1], b = WHOLE ? S.total : S.offq[k * S.ncol + m + 2];
        for (int base = a; base < b; base += 32) {
          const int j = base + lane;
          bool in = false;
          if (j < b && j != l && (!HALF || sh_gid[j] > gi))
            in = candidate_in<MIXED, WHOLE>(smem, L, l, j, x, N, g, band);
          const unsigned msk = __ballot_sync(0xffffffffu, in);
          if (lane == 0 && c < ta.max_chunks) masks[o * ta.max_chunks + c] = msk;
          ++c;
          cnt += __popc(msk);
        }
      }
      if (lane == 0) s_cnt[o] = (c <= ta.max_chunks) ? cnt : -1;
    }
    __syncthreads();
    if (warp == 0) {
      // exclusive prefix of the row sizes; one atomic reserves the tile's segment, padded to a
      // multiple of 8 entries (16 bytes) so that the force kernel can bulk-copy it
      unsigned run = 0;
      bool ok = true;
      for (int base = 0; base < n_own; base += 32) {
        const int o = base + lane;
        const int v0 = o < n_own ? s_cnt[o] : 0;
        ok = ok && __all_sync(0xffffffffu, v0 >= 0);
        const unsigned v = v0 > 0 ? (unsigned)v0 : 0u;
        unsigned inc = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const unsigned y = __shfl_up_sync(0xffffffffu, inc, d);
          if (lane >= d) inc += y;
        }
        if (o < n_own) s_pre[o] = (int)(run + inc - v);
        run += __shfl_sync(0xffffffffu, inc, 31);
      }
      if (lane == 0) {
        const unsigned padded = (run + 7u) & ~7u;
        const unsigned long long b = atomicAdd(counter, (unsigned long long)padded);
        atomicAdd(counter + 1, (unsigned long long)run);
        const bool fits = ok && (b + padded <= cap);
        s_base = (unsigned)b;
        s_ok = fits;
        tile_list[t] = fits ? make_uint2((unsigned)b, padded) : make_uint2(0u, 0u);
        atomicMax(max_list, padded);
        if (!ok) atomicOr(status, LJ_ST_CELL_RANGE);
      }
    }
    __syncthreads();
    // phase 2: rows and entries
    for (int o = warp; o < n_own; o += kWarps) {
      const int l = S.own0 + o;
      const int gi = sh_gid[l];
      const int m = WHOLE ? 0 : own_cell(S, l, ti.Tp);
      const unsigned start = s_base + (unsigned)s_pre[o];
      if (lane == 0) rows[gi] = s_ok ? make_uint2(start, (unsigned)s_cnt[o]) : make_uint2(0u, 0u);
      if (!s_ok) continue;
      unsigned p = start;
      int c = 0;
      for (int k = 0; k < nk; ++k) {
        const int a = WHOLE ? 0 : S.offq[k * S.ncol + m - 1], b = WHOLE ? S.total : S.offq[k * S.ncol + m + 2];
        for (int base = a; base < b; base += 32) {
          const unsigned msk = masks[o * ta.max_chunks + c];
          ++c;
          if ((msk >> lane) & 1u) ent[p + __popc(msk & lt)] = (uint16_t)(base + lane);
          p += __popc(msk);
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// Pair-list construction by cell windows (staged tiles, both forms, both list kinds).
//
// The keys of a tile are taken 32 at a time (a group, one key per lane, consecutive in the cell
// order, so a group spans two or three own cells).  A work item is (group, neighbour column k):
// every lane tests its own key against the three cells m-1, m, m+1 of column k around its own
// cell m (the window of Alg. 1: partners farther along z fail the distance test, cells being at
// least r_s wide).  Lanes in one cell read the same staged record, so a load serves a group with
// one or a few distinct addresses.  The kept-candidate bits of each 32-candidate word go to a
// per-tile pool in shared memory; a count per (key, column) gives every key its row and each
// column its place in the row (columns in order, partners ascending: the list is deterministic);
// one atomic reserves the tile's segment (padded to 8 entries) while the entries are written from
// the bits into shared memory over the staged positions (no longer needed) and then copied out
// with 16-byte stores.  Items whose bits do not fit in the pool are tested again when written (and
// that tile's entries go to global memory directly).  Warp 0 takes the next tile's bookkeeping while
// the others count, its cell bounds copied a tile ahead with cp.async.  With the half list, a
// column other than the key's own has all its cells before or all after the key's in the cell
// order (cell = (X n + Y) n + Z), so such a column is kept or skipped as a whole; in the own column
// the sorted indices decide per pair.
constexpr int kWinPoolPerItem = 2;  // pool words per work item on average (two words hold 64 candidates)
constexpr int kWinThreads = 256;    // threads of a window-kernel CTA
constexpr int kWinCtas = 3;         // window-kernel CTAs resident per SM (register budget)

struct WinLayout {
  size_t pos;    // hi float4 [max_staged + 32] (w: sorted index bits; 32 slack records for the last word);
                 // once the bits are taken, the tile's segment (uint16 [seg_cap]) before it is copied out
  size_t cell;   // uint8 [max_own]: own cell (1..Tp) of each key
  size_t cnt;    // uint16 [ngrp * 9 * 32]: per (key, column) count, then its offset in the key's row
  size_t kst;    // int [max_own]: row start in the segment; then int [max_own]: row length
  size_t ib;     // int [ngrp * 9]: first pool word of each item (-1: tested again when written)
  size_t gtot;   // int [ngrp]: entries of each group of 32 keys
  size_t mask;   // uint32 [pool_words * 32]
  int ngrp, pool_words, seg_cap;
  size_t total;
};

__host__ __device__ __forceinline__ WinLayout win_layout(const TileArgs& ta) {
  WinLayout W;
  const size_t ms = (size_t)ta.max_staged + 32;
  W.ngrp = (ta.max_own + 31) / 32;
  W.pos = 0;
  size_t o = align16(ms * 16);
  W.seg_cap = (int)((ms * 8) & ~(size_t)7);
  W.cell = o;
  o += align16((size_t)ta.max_own);
  W.cnt = o;
  o += align16((size_t)W.ngrp * 9 * 32 * 2);
  W.kst = o;
  o += align16((size_t)ta.max_own * 8);
  W.ib = o;
  o += align16((size_t)W.ngrp * 9 * 4);
  W.gtot = o;
  o += align16((size_t)W.ngrp * 4);
  W.pool_words = W.ngrp * 9 * kWinPoolPerItem + 8;
  W.mask = o;
  o += (size_t)W.pool_words * 32 * 4;
  W.total = o;
  return W;
}

// Order of neighbour column k against the tile's own column, for the half list: +1 if all cells of
// column k come after the tile's own cells in the cell order, -1 if all come before, 0 for the own
// column (decided per pair by the sorted indices).
__device__ __forceinline__ int win_column_order(const TileInfo& ti, int n, int k) {
  if (k == 4) return 0;
  int sx, sy;
  const int X = wrap_cell(ti.cx + k / 3 - 1, n, sx);
  const int Y = wrap_cell(ti.cy + k % 3 - 1, n, sy);
  return (X > ti.cx || (X == ti.cx && Y > ti.cy)) ? 1 : -1;
}

// One 32-candidate word of a key: bit u set iff staged slot jb + u is listed for the key (slot l,
// sorted index gi, hi record pi).  `rem` candidates of the key remain from jb on (the rest of the
// word is masked); lanes without any read slots 0..31 and keep nothing.  Only the first nblk blocks of
// 8 candidates are tested (the windows of all lanes end before the rest).  FP32 filter on the exact
// hi differences; for a word with a kept r^2 inside the band the FP64 test of the oracle decides
// those.  OWN: the key's own column (the key itself is dropped; HALF keeps larger sorted indices).
template <bool HALF, bool OWN>
__device__ __forceinline__ uint32_t win_word(const float4* sh_pos, const double* __restrict__ x, int64_t N,
                                             const Geom& g, const ListBand& band, int jb, int rem, int nblk, int l,
                                             int gi, float4 pi) {
  uint32_t bits = 0;
  float mx = 0.f;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    if (b >= nblk) break;  // warp-uniform: blocks of 8 past every lane's window are not tested
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const int u = 8 * b + v;
      const float4 pj = sh_pos[jb + u];
      const float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;  // exact
      const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      bool in = r2 < band.hi;
      if (HALF && OWN) in = in && __float_as_int(pj.w) > gi;
      if (in) {
        bits |= 1u << u;
        mx = fmaxf(mx, r2);
      }
    }
  }
  bits &= rem >= 32 ? 0xffffffffu : (rem > 0 ? (1u << rem) - 1u : 0u);
  if (OWN) {
    const int d = l - jb;
    if (d >= 0 && d < 32) bits &= ~(1u << d);  // the key itself
  }
  const bool band_hit = bits != 0u && mx >= band.lo;
  if (__any_sync(0xffffffffu, band_hit) && band_hit) {
    uint32_t mb = bits;
    while (mb) {
      const int u = __ffs(mb) - 1;
      mb &= mb - 1;
      const float4 pj = sh_pos[jb + u];
      const float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
      const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      if (r2 >= band.lo && !pair_in_exact(x, N, gi, __float_as_int(pj.w), g, band.rs2)) bits &= ~(1u << u);
    }
  }
  return bits;
}

template <bool HALF>
__device__ __forceinline__ uint32_t win_word_k(bool own, const float4* sh_pos, const double* __restrict__ x,
                                               int64_t N, const Geom& g, const ListBand& band, int jb, int rem,
                                               int nblk, int l, int gi, float4 pi) {
  return own ? win_word<HALF, true>(sh_pos, x, N, g, band, jb, rem, nblk, l, gi, pi)
             : win_word<HALF, false>(sh_pos, x, N, g, band, jb, rem, nblk, l, gi, pi);
}

size_t list_smem_bytes(const TileArgs& ta, int precision) {
  if (!ta.whole) return win_layout(ta).total;  // both forms: the FP32 filter on the hi copies
  return tile_layout(ta, precision == LJ_MIXED, false).total;
}

template <bool HALF, bool BATCHED, int NT>
__global__ void __launch_bounds__(NT, kWinCtas)
    k_list_win(const float4* __restrict__ pos, const double* __restrict__ x, const uint32_t* __restrict__ cs_in,
               int64_t N, Geom g_in, TileArgs ta_in, ListBand band, uint2* __restrict__ rows,
               uint2* __restrict__ tile_list, uint16_t* __restrict__ ent, uint64_t cap,
               unsigned long long* __restrict__ counter, unsigned int* __restrict__ max_list,
               int32_t* __restrict__ status, const ReplicaGeo* __restrict__ reps, int R,
               const int* __restrict__ pred, const int32_t* __restrict__ tile_rep) {
  static_assert(NT >= 64, "warp 0 prepares the next tile while the others count");
  if (pred && !*pred) return;  // predicated (batched rebuild inside a graph)
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ TileShared Sb[2];  // bookkeeping of the current tile and of the next one
  __shared__ __align__(8) uint64_t bar;
  __shared__ unsigned int s_base;
  __shared__ int s_fits, s_pool, s_retest;
  __shared__ int s_ready[2];  // the buffer's tile fits the capacities
  constexpr int kNW = NT / 32;
  const WinLayout W = win_layout(ta_in);
  TileLayout L;  // the staging helpers' view: hi records (sorted indices in w)
  L.pos = W.pos;
  L.gid = W.pos;
  L.rows = L.ent = L.cnt = L.total = 0;
  const float4* sh_pos = (const float4*)(smem + W.pos);
  unsigned char* s_cell = smem + W.cell;
  uint16_t* s_cnt = (uint16_t*)(smem + W.cnt);
  int* s_kst = (int*)(smem + W.kst);
  int* s_len = s_kst + ta_in.max_own;
  int* s_ib = (int*)(smem + W.ib);
  int* s_gtot = (int*)(smem + W.gtot);
  uint32_t* s_mask = (uint32_t*)(smem + W.mask);
  uint16_t* s_seg = (uint16_t*)(smem + W.pos);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t phase = 0;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_proxy_async_smem();
  }
  __shared__ uint32_t s_pfa[kMaxCells], s_pfb[kMaxCells];  // cell bounds of the tile being prefetched
  TileInfo pf_ti;  // warp 0: that tile
  auto prefetch = [&](int64_t tp) {  // warp 0: a tile's cell bounds, copied a tile ahead of their use
    TileArgs tap = ta_in;
    Geom gp = g_in;
    const uint32_t* csp = cs_in;
    int64_t tlp = tp;
    if (BATCHED) {
      const ReplicaGeo& rg = reps[tile_rep[tp]];
      replica_view(rg, tap, gp);
      csp = cs_in + rg.cell_base;
      tlp = tp - rg.tile_base;
    }
    pf_ti = tile_info(tlp, tap);
    tile_prefetch_async(pf_ti, tap, csp, s_pfa, s_pfb, lane);
  };
  auto prepare = [&](int b) {  // warp 0: buffer b from the prefetched bounds
    const bool okp = tile_prepare_async(pf_ti, s_pfa, s_pfb, ta_in, Sb[b], lane);
    if (lane == 0) s_ready[b] = (okp && Sb[b].own1 - Sb[b].own0 <= ta_in.max_own) ? 1 : 0;
  };
  if (warp == 0 && blockIdx.x < ta_in.ntiles) {
    prefetch(blockIdx.x);
    prepare(0);
    if (blockIdx.x + gridDim.x < ta_in.ntiles) prefetch(blockIdx.x + gridDim.x);
  }
  __syncthreads();

  int buf = 0;
  for (int64_t t = blockIdx.x; t < ta_in.ntiles; t += gridDim.x, buf ^= 1) {
    TileShared& S = Sb[buf];
    TileArgs ta = ta_in;
    Geom g = g_in;
    int64_t tl = t;
    if (BATCHED) {  // the tile's replica: its box, grid and cells
      const ReplicaGeo& rg = reps[tile_rep[t]];
      replica_view(rg, ta, g);
      tl = t - rg.tile_base;
    }
    const TileInfo ti = tile_info(tl, ta);
    auto prepare_next = [&]() {  // warp 0
      if (t + gridDim.x < ta_in.ntiles) {
        prepare(buf ^ 1);
        if (t + 2 * (int64_t)gridDim.x < ta_in.ntiles) prefetch(t + 2 * (int64_t)gridDim.x);
      }
    };
    if (!s_ready[buf]) {  // sizing inconsistency: record and skip the tile
      if (threadIdx.x == 0) atomicOr(status, LJ_ST_CELL_RANGE);
      if (warp == 0) prepare_next();
      __syncthreads();
      continue;
    }
    if (threadIdx.x == 0) {
      s_pool = 0;
      s_retest = 0;
    }
    const int n_own = S.own1 - S.own0, ncol = S.ncol;
    // own cell of every key (ordered before the staged records by the barrier that ends the wait)
    for (int m = 1 + warp; m <= ti.Tp; m += kNW) {
      const int a = S.offq[4 * ncol + m] - S.own0, b = S.offq[4 * ncol + m + 1] - S.own0;
      for (int o = a + lane; o < b; o += 32) s_cell[o] = (unsigned char)m;
    }
    stage_issue<true, false>(ti, ta, pos, nullptr, nullptr, S, smem, L, &bar);
    if (!stage_finish<true, false>(ti, ta, g, S, smem, L, &bar, phase, false, status)) return;
    const int ngrp = (n_own + 31) >> 5, nitem = 9 * ngrp;
    // phase A: the kept-candidate bits of every item, a count per (key, column)
    for (int item = warp; item < nitem; item += kNW) {
      const int gq = item / 9, k = item - 9 * gq;
      const int o = 32 * gq + lane;
      const bool valid = o < n_own;
      const int oc = valid ? o : n_own - 1;
      const int l = S.own0 + oc;
      const float4 pi = sh_pos[l];
      const int gi = __float_as_int(pi.w);
      const int m = s_cell[oc];
      const int j0 = S.offq[k * ncol + m - 1];
      int len = valid ? S.offq[k * ncol + m + 2] - j0 : 0;
      if (HALF && win_column_order(ti, ta.n, k) < 0) len = 0;
      const int maxlen = __reduce_max_sync(0xffffffffu, len);
      const int nw = (maxlen + 31) >> 5;
      int base = 0;
      if (lane == 0) {
        base = nw > 0 ? atomicAdd(&s_pool, nw) : 0;
        if (base + nw > W.pool_words) {
          base = -1;
          s_retest = 1;
        }
        s_ib[item] = base;
      }
      base = __shfl_sync(0xffffffffu, base, 0);
      int cnt = 0;
      for (int w = 0; w < nw; ++w) {
        const int rem = len - 32 * w;
        const uint32_t bits = win_word_k<HALF>(k == 4, sh_pos, x, N, g, band, rem > 0 ? j0 + 32 * w : 0, rem,
                                               (maxlen - 32 * w + 7) >> 3, l, gi, pi);
        if (base >= 0) s_mask[(base + w) * 32 + lane] = bits;
        cnt += __popc(bits);
      }
      s_cnt[item * 32 + lane] = (uint16_t)cnt;
    }
    __syncthreads();
    // phase B (warps 1..): each key's column offsets within its row, its row length and its row's
    // place within its group of 32 keys; the group's entries.  Warp 0 meanwhile takes the next
    // tile's bookkeeping.
    if (warp == 0) prepare_next();
    for (int gq = warp - 1; gq >= 0 && gq < ngrp; gq += kNW - 1) {
      int run = 0;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        uint16_t* c = s_cnt + (9 * gq + k) * 32 + lane;
        const int v = *c;
        *c = (uint16_t)run;
        run += v;
      }
      const int o = 32 * gq + lane;
      const int v = o < n_own ? run : 0;
      int inc = v;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
      }
      if (o < n_own) {
        s_len[o] = run;
        s_kst[o] = inc - v;
      }
      if (lane == 31) s_gtot[gq] = inc;
    }
    __syncthreads();
    // the tile's entries (every thread); one atomic reserves its segment, padded to 8 entries
    int total = 0;
    for (int gq = 0; gq < ngrp; ++gq) total += s_gtot[gq];
    const unsigned padded = ((unsigned)total + 7u) & ~7u;
    const bool staged = padded <= (unsigned)W.seg_cap && !s_retest;
    if (threadIdx.x == 0) {
      const unsigned long long b = atomicAdd(counter, (unsigned long long)padded);
      atomicAdd(counter + 1, (unsigned long long)total);
      const bool fits = b + padded <= cap;
      s_base = (unsigned)b;
      s_fits = fits;
      tile_list[t] = fits ? make_uint2((unsigned)b, padded) : make_uint2(0u, 0u);
      atomicMax(max_list, padded);
      if (BATCHED && !fits) atomicOr(status, LJ_ST_LIST_OVERFLOW);  // no host retry inside a graph
    }
    // phase D: the entries of every item from its bits (or tested again), in row order; staged
    // over the positions (no longer needed unless an item is tested again) and copied out, or
    // written to global memory directly once the segment's place is known
    auto write_items = [&](auto in_shared) {
      uint16_t* dst = decltype(in_shared)::value ? s_seg : ent + s_base;
      for (int item = warp; item < nitem; item += kNW) {
        const int gq = item / 9, k = item - 9 * gq;
        const int o = 32 * gq + lane;
        const bool valid = o < n_own;
        const int oc = valid ? o : n_own - 1;
        const int m = s_cell[oc];
        const int j0 = S.offq[k * ncol + m - 1];
        int len = valid ? S.offq[k * ncol + m + 2] - j0 : 0;
        if (HALF && win_column_order(ti, ta.n, k) < 0) len = 0;
        int gbase = 0;
        for (int q = 0; q < gq; ++q) gbase += s_gtot[q];
        int p = valid ? gbase + s_kst[o] + s_cnt[item * 32 + lane] : 0;
        const int base = s_ib[item];
        if (base >= 0) {
          for (int w = 0; 32 * w < len; ++w) {
            uint32_t bits = s_mask[(base + w) * 32 + lane];
            while (bits) {
              const int u = __ffs(bits) - 1;
              bits &= bits - 1;
              dst[p++] = (uint16_t)(j0 + 32 * w + u);
            }
          }
        } else if (!decltype(in_shared)::value) {
          const int l = S.own0 + oc;
          const float4 pi = sh_pos[l];
          const int gi = __float_as_int(pi.w);
          const int maxlen = __reduce_max_sync(0xffffffffu, len);
          const int nw = (maxlen + 31) >> 5;
          for (int w = 0; w < nw; ++w) {
            const int rem = len - 32 * w;
            uint32_t bits = win_word_k<HALF>(k == 4, sh_pos, x, N, g, band, rem > 0 ? j0 + 32 * w : 0, rem,
                                             (maxlen - 32 * w + 7) >> 3, l, gi, pi);
            while (bits) {
              const int u = __ffs(bits) - 1;
              bits &= bits - 1;
              dst[p++] = (uint16_t)(j0 + 32 * w + u);
            }
          }
        }
      }
    };
    if (staged) {
      write_items(std::true_type());
      __syncthreads();
    } else {
      __syncthreads();
      if (s_fits) write_items(std::false_type());
    }
    const bool fits = s_fits != 0;
    for (int o = threadIdx.x; o < n_own; o += NT) {
      int gbase = 0;
      for (int q = 0; q < (o >> 5); ++q) gbase += s_gtot[q];
      rows[S.gown0 + o] = fits ? make_uint2(s_base + (unsigned)(gbase + s_kst[o]), (unsigned)s_len[o]) : make_uint2(0u, 0u);
    }
    if (staged && fits) {
      const uint4* src = (const uint4*)s_seg;
      uint4* out = (uint4*)(ent + s_base);
      for (unsigned w = threadIdx.x; w < padded / 8u; w += NT) out[w] = src[w];
    }
    // the positions' bytes were read and written by the generic proxy; the next tile's bulk copies
    // (async proxy) write them
    fence_proxy_async_smem();
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
template <int LANES>
__device__ __forceinline__ float gsum(float v) {
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <int LANES>
__device__ __forceinline__ double gsum(double v) {
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Shared memory of the force kernel: `nbuf` tile buffers (with two, the next tile's copies are in
// flight while the current one is computed); one for the whole-box case.
size_t force_buffer_bytes(const TileArgs& ta, int precision, int half) {
  const bool mixed = precision == LJ_MIXED;
  return align16(tile_layout(ta, mixed, true, !mixed && (half || ta.whole)).total);
}
size_t force_smem_bytes(const TileArgs& ta, int precision, int nbuf, int half) {
  return (ta.whole ? 1 : (nbuf == 2 ? 2 : 1)) * force_buffer_bytes(ta, precision, half);
}

// 1/x from the hardware approximation (rcp.approx) refined by one Newton-Raphson step
// r' = r + r (1 - x r), which roughly squares its relative error.
__device__ __forceinline__ float rcp_nr(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return fmaf(r, fmaf(-x, r, 1.0f), r);
}

// 1/x in FP64 from the hardware approximation (rcp.approx.ftz.f64) refined by two Newton-Raphson
// steps r' = r + r (1 - x r), each of which squares the relative error: full double precision to
// within an ulp, in a handful of FP64 operations instead of a correctly rounded reciprocal.
__device__ __forceinline__ double rcp_nr64(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  r = fma(r, fma(-x, r, 1.0), r);
  return fma(r, fma(-x, r, 1.0), r);
}

struct AccF {
  float fx, fy, fz, pe, vir;
};

// Per-thread energy and virial sums over the keys a thread finishes: FP32 partials of at most
// 16 keys, folded into FP64 totals (so the FP64 pipe, 1/64 of the FP32 rate on this part, sees one
// add per 16 keys).  The mixed form's virial partial is in units of 1/u and is scaled by u
// (exactly: u = 2^-qk) when folded.
struct EAcc {
  double pe = 0.0, vir = 0.0;
  float pe32 = 0.0f, vir32 = 0.0f;
  int n = 0;
  float vscale = 1.0f;
  __device__ __forceinline__ void flush() {
    pe += (double)pe32;
    vir += (double)(vir32 * vscale);
    pe32 = vir32 = 0.0f;
    n = 0;
  }
  __device__ __forceinline__ void add32(float p, float v) {
    pe32 += p;
    vir32 += v;
    if (++n == 16) flush();
  }
};

// Partner difference of two fixed-point records in units of u: the exact integer difference
// converted once to FP32.  WHOLE: the nearest periodic image is chosen per pair (the raw
// difference is below 2^31 u there) and round(L / u) subtracted as an integer.
template <bool WHOLE>
__device__ __forceinline__ float qd(uint32_t a, uint32_t b, const Geom& g) {
  int d = (int)(a - b);
  if (WHOLE) d -= (int)rintf(__int2float_rn(d) * g.q_inv_L) * (int)g.Lq;
  return __int2float_rn(d);
}

// One listed pair in the mixed form (Alg. 6 in eps/sigma form) on differences in units of u:
//   f = ri2 s3i (24 eps - 48 eps s3i) + 8 eps c2 / sigma^2, zero for r^2 >= r_c^2 (select)
//   V = 4 eps [s3i (s3i - 1) + c2 r^2 / sigma^2 + c0],  W += -f r^2
// with the constants scaled by powers of u (LJConst::*q), so f d and V come out in sigma units and
// W in units of 1/u.  HALF: Newton-3 scatter to the partner's sorted index, carried in qj.w.
template <bool HALF, bool ENERGY, bool WHOLE>
__device__ __forceinline__ void pair_q(const uint4& qi, const uint4& qj, const LJConst& c, const Geom& g, AccF& a,
                                       float4* fout) {
  const float dx = qd<WHOLE>(qj.x, qi.x, g), dy = qd<WHOLE>(qj.y, qi.y, g), dz = qd<WHOLE>(qj.z, qi.z, g);
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const float ri2 = rcp_nr(r2);
  const float si = c.sig2q * ri2;
  const float s3i = si * si * si;
  const bool in = r2 < c.rc2q;
  float ff = fmaf(ri2 * s3i, fmaf(-c.f48q, s3i, c.f24q), c.f8c2q);
  ff = in ? ff : 0.0f;
  a.fx = fmaf(ff, dx, a.fx);
  a.fy = fmaf(ff, dy, a.fy);
  a.fz = fmaf(ff, dz, a.fz);
  if (HALF) atomicAdd(&fout[qj.w], make_float4(-ff * dx, -ff * dy, -ff * dz, 0.0f));
  if (ENERGY) {
    const float v = c.e4 * fmaf(s3i, s3i - 1.0f, fmaf(c.c2q, r2, c.c0f));
    a.pe += in ? v : 0.0f;
    a.vir = fmaf(-ff, r2, a.vir);
  }
}

// Forces of the own particles of one staged tile (buffer `buf`); group `grp` of LANES threads per
// key particle, lanes striding over its row.
template <bool MIXED, int LANES, bool HALF, bool ENERGY, bool WHOLE, bool LONGLIST, int NTH = kTileThreads>
__device__ __forceinline__ void force_tile_compute(const TileShared& S, const unsigned char* buf, const TileLayout& L,
                                                   const uint2* __restrict__ rows, const uint16_t* __restrict__ ent,
                                                   const LJConst& c, const Geom& g, void* __restrict__ fout,
                                                   int32_t* __restrict__ status, EAcc& eacc, int list_cap) {
  const void* sh_pos = buf + L.pos;
  const int* sh_gid = (const int*)(buf + L.gid);
  const uint2* s_rows = (const uint2*)(buf + L.rows);
  const uint16_t* s_ent = (const uint16_t*)(buf + L.ent);
  const int lane = threadIdx.x & (LANES - 1);
  const int grp = threadIdx.x / LANES;
  constexpr int kGroups = NTH / LANES;  // groups of the computing threads
  const double f24d = 24.0 * c.eps, f48d = 48.0 * c.eps, f8c2d = 8.0 * c.eps * c.c2 / c.sig2;
  const double e4d = 4.0 * c.eps, c2sd = c.c2 / c.sig2;
  const int n_own = S.own1 - S.own0;
  for (int o = grp; __any_sync(0xffffffffu, o < n_own); o += kGroups) {
    const bool valid = o < n_own;
    AccF a0{0.f, 0.f, 0.f, 0.f, 0.f}, a1{0.f, 0.f, 0.f, 0.f, 0.f};
    double dfx = 0.0, dfy = 0.0, dfz = 0.0, dpe = 0.0, dvir = 0.0;
    int gi = 0;
    if (valid) {
      const int l = S.own0 + o;
      gi = S.gown0 + o;
      uint2 row;
      if (WHOLE) {
        row = rows[gi];
      } else {
        row = s_rows[S.row_off + o];
        row.x -= S.list_base;
        if (row.x + row.y > S.list_len) {  // inconsistent row: record and skip
          if (lane == 0) atomicOr(status, LJ_ST_LIST_OVERFLOW);
          row.y = 0;
        }
      }
      // the row's pairs; one instance per memory space of the list (in_smem: staged segment)
      auto row_pairs = [&](const uint16_t* __restrict__ el, bool in_smem) {
      if (MIXED) {
        // staged fixed-point records by 32-bit shared address: record j at a_pos + 16 j
        const uint32_t a_pos = smem_addr(sh_pos);
        const uint4 qi = lds_u4(a_pos + 16u * l);
        float4* F = (float4*)fout;
        auto pair_at = [&](uint32_t j, AccF& acc) {
          pair_q<HALF, ENERGY, WHOLE>(qi, lds_u4(a_pos + (j << 4)), c, g, acc, F);
        };
        if (in_smem) {
          // list segment staged: entries by 32-bit shared address, two independent per iteration
          uint32_t p = smem_addr(s_ent) + 2u * (row.x + lane);
          const uint32_t pend = smem_addr(s_ent) + 2u * (row.x + row.y);
          for (; p + 2u * LANES < pend; p += 4u * LANES) {
            const uint32_t j0 = lds_u16(p), j1 = lds_u16(p + 2u * LANES);
            pair_at(j0, a0);
            pair_at(j1, a1);
          }
          if (p < pend) pair_at(lds_u16(p), a0);
        } else {
          unsigned e = lane;
          for (; e + LANES < row.y; e += 2 * LANES) {
            const uint32_t j0 = el[row.x + e], j1 = el[row.x + e + LANES];
            pair_at(j0, a0);
            pair_at(j1, a1);
          }
          if (e < row.y) pair_at(el[row.x + e], a0);
        }
      } else {
        const dvec4 qi = ((const dvec4*)sh_pos)[l];
        for (unsigned e = lane; e < row.y; e += LANES) {
          const int j = el[row.x + e];
          const dvec4 qj = ((const dvec4*)sh_pos)[j];  // its image already in place (tiles)
          double dx = qj.x - qi.x, dy = qj.y - qi.y, dz = qj.z - qi.z;
          if (WHOLE) {
            dx = fma(-rint(dx * g.inv_L64), g.L, dx);
            dy = fma(-rint(dy * g.inv_L64), g.L, dy);
            dz = fma(-rint(dz * g.inv_L64), g.L, dz);
          }
          const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
          const double ri2 = rcp_nr64(r2);
          const double si = c.sig2 * ri2;
          const double s3i = si * si * si;
          const bool in = r2 < c.rc2;
          double ff = fma(ri2 * s3i, fma(-f48d, s3i, f24d), f8c2d);
          ff = in ? ff : 0.0;
          dfx = fma(ff, dx, dfx);
          dfy = fma(ff, dy, dfy);
          dfz = fma(ff, dz, dfz);
          if (HALF) {
            dvec4* F = (dvec4*)fout;
            const int gj = sh_gid[j];
            atomicAdd(&F[gj].x, -ff * dx);
            atomicAdd(&F[gj].y, -ff * dy);
            atomicAdd(&F[gj].z, -ff * dz);
          }
          if (ENERGY) {
            const double v = e4d * fma(s3i, s3i - 1.0, fma(c2sd, r2, c.c0));
            dpe += in ? v : 0.0;
            dvir = fma(-ff, r2, dvir);
          }
        }
      }
      };
      if (WHOLE) row_pairs(ent, false);
      else if (!LONGLIST || S.list_len <= (unsigned)list_cap) row_pairs(s_ent, true);
      else row_pairs(ent + S.list_base, false);  // a long segment stays in HBM
    }
    if (MIXED) {
      float fx = gsum<LANES>(a0.fx + a1.fx);
      float fy = gsum<LANES>(a0.fy + a1.fy);
      float fz = gsum<LANES>(a0.fz + a1.fz);
      if (valid && lane == 0) {
        if (HALF) atomicAdd(&((float4*)fout)[gi], make_float4(fx, fy, fz, 0.0f));
        else ((float4*)fout)[gi] = make_float4(fx, fy, fz, 0.0f);
      }
      if (ENERGY) {  // the group's lanes reduce in FP32, one lane accumulates
        const float pe = gsum<LANES>(a0.pe + a1.pe), vir = gsum<LANES>(a0.vir + a1.vir);
        if (lane == 0) eacc.add32(pe, vir);
      }
    } else {
      dfx = gsum<LANES>(dfx);
      dfy = gsum<LANES>(dfy);
      dfz = gsum<LANES>(dfz);
      if (valid && lane == 0) {
        dvec4* F = (dvec4*)fout;
        if (HALF) {
          atomicAdd(&F[gi].x, dfx);
          atomicAdd(&F[gi].y, dfy);
          atomicAdd(&F[gi].z, dfz);
        } else {
          F[gi] = make_dvec4(dfx, dfy, dfz, 0.0);
        }
      }
      if (ENERGY) {
        eacc.pe += dpe;
        eacc.vir += dvir;
      }
    }
  }
}

// Bookkeeping of one tile before its copies are issued: segment of the list, cell bounds,
// capacity checks (identical in every thread).  Returns whether the tile can be staged.
__device__ __forceinline__ bool force_tile_prepare(const TileInfo& ti, int64_t t, const TileArgs& ta,
                                                   const uint32_t* __restrict__ cs,
                                                   const uint2* __restrict__ tile_list, TileShared& S,
                                                   int32_t* __restrict__ status) {
  if (threadIdx.x == blockDim.x - 1) {
    const uint2 tl = tile_list[t];
    S.list_base = tl.x;
    S.list_len = tl.y;
  }
  if (!stage_offsets(ti, ta, cs, S)) {
    if (threadIdx.x == 0) atomicOr(status, LJ_ST_CELL_RANGE);
    return false;
  }
  if (S.own1 - S.own0 > ta.max_own || S.list_len > (unsigned)ta.max_list) {
    if (threadIdx.x == 0) atomicOr(status, LJ_ST_LIST_OVERFLOW);
    return false;
  }
  return true;
}

// Force over the list, tile by tile.  With nbuf = 2 each CTA walks its tiles with two
// shared-memory buffers: the copies of tile t + gridDim.x are issued before tile t is computed,
// so the copy latency overlaps the pair arithmetic; with nbuf = 1 the tiles are staged one after
// the other and the overlap comes from the other CTAs of the SM.  Energies: per-thread FP64
// sums -> one partial per block.
template <bool MIXED, int LANES, bool HALF, bool ENERGY, bool WHOLE, bool LONGLIST>
__global__ void __launch_bounds__(kTileThreads, 4)
    k_force_tile(const void* __restrict__ pos, const uint32_t* __restrict__ cs, int64_t N, Geom g, TileArgs ta,
                 LJConst c, const uint2* __restrict__ rows, const uint2* __restrict__ tile_list,
                 const uint16_t* __restrict__ ent, void* __restrict__ fout, double* __restrict__ part,
                 int32_t* __restrict__ status, int nbuf, const int* __restrict__ skip) {
  if (skip && *skip) return;  // a device-decided run stopped before this step
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ TileShared SS[2];
  __shared__ __align__(8) uint64_t bars[2];
  const TileLayout L = tile_layout(ta, MIXED, true, !MIXED && (HALF || WHOLE));
  const size_t buf_bytes = align16(L.total);
  EAcc eacc;
  eacc.vscale = g.qu;
  if (WHOLE) {
    if (blockIdx.x == 0) {
      stage_whole<MIXED, !MIXED>(N, pos, SS[0], smem, L);
      __syncthreads();
      force_tile_compute<MIXED, LANES, HALF, ENERGY, true, false>(SS[0], smem, L, rows, ent, c, g, fout, status, eacc,
                                                                  ta.list_cap);
    }
  } else {
    const bool pipelined = nbuf == 2;
    if (threadIdx.x == 0) {
      mbar_init(&bars[0], 1);
      mbar_init(&bars[1], 1);
      fence_proxy_async_smem();
    }
    __syncthreads();
    uint32_t ph0 = 0, ph1 = 0;
    int64_t t = blockIdx.x;
    int b = 0;
    bool v_cur = false, v_next = false;
    if (pipelined && t < ta.ntiles) {
      v_cur = force_tile_prepare(tile_info(t, ta), t, ta, cs, tile_list, SS[0], status);
      if (v_cur) stage_issue<MIXED, true>(tile_info(t, ta), ta, pos, rows, ent, SS[0], smem, L, &bars[0]);
    }
    for (; t < ta.ntiles; t += gridDim.x) {
      if (!pipelined) {
        v_cur = force_tile_prepare(tile_info(t, ta), t, ta, cs, tile_list, SS[0], status);
        if (v_cur) stage_issue<MIXED, true>(tile_info(t, ta), ta, pos, rows, ent, SS[0], smem, L, &bars[0]);
      } else {
        const int64_t tn = t + gridDim.x;
        v_next = false;
        if (tn < ta.ntiles) {
          v_next = force_tile_prepare(tile_info(tn, ta), tn, ta, cs, tile_list, SS[b ^ 1], status);
          if (v_next)
            stage_issue<MIXED, true>(tile_info(tn, ta), ta, pos, rows, ent, SS[b ^ 1], smem + (b ^ 1) * buf_bytes, L,
                                     &bars[b ^ 1]);
        }
      }
      if (v_cur) {
        uint32_t& ph = b ? ph1 : ph0;
        if (!stage_finish<MIXED, true>(tile_info(t, ta), ta, g, SS[b], smem + b * buf_bytes, L, &bars[b], ph,
                                       !MIXED && HALF, status)) {
          if (v_next) mbar_wait(&bars[b ^ 1], b ? ph0 : ph1, kWaitBudget);  // drain the other buffer's copies
          return;
        }
        force_tile_compute<MIXED, LANES, HALF, ENERGY, false, LONGLIST>(SS[b], smem + b * buf_bytes, L, rows, ent, c, g,
                                                                        fout, status, eacc, ta.list_cap);
      }
      __syncthreads();
      if (pipelined) {
        v_cur = v_next;
        b ^= 1;
      }
    }
  }
  if (ENERGY) {
    __shared__ double sh[32];
    eacc.flush();
    const double tp = block_sum(eacc.pe, sh);
    __syncthreads();
    const double tv = block_sum(eacc.vir, sh);
    if (threadIdx.x == 0) {
      part[2 * (size_t)blockIdx.x] = tp;
      part[2 * (size_t)blockIdx.x + 1] = tv;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Pipelined force (mixed form, full list, tiled box): two producer warps stage tiles into two
// shared-memory buffers (producer p handles the tiles k = p mod 2, in buffer p) while the consumer
// warps compute, so neither the copies nor the tile-end stragglers hold the CTA at a barrier.
// Per tile k (buffer k % 2, bookkeeping slot k % 4):
//   producer: wait empty[b] (tile k - 2 released) -> issue the copies of tile k -> bookkeeping of
//             tile k + 2 from cell bounds loaded one tile earlier, and the loads for tile k + 4 ->
//             wait full[b] -> arrive ready[b];
//   consumers: wait ready[b] -> (periodic tiles: image shifts, consumer barrier) -> forces of
//             the tile's own particles -> arrive empty[b].
// Every wait is bounded; a producer that gives up marks the slot aborted and releases the
// consumers, which then leave.  No copy is in flight when a warp leaves.
constexpr int kPipeProducers = 2;
constexpr int kPipeSlots = 4;
__host__ __device__ constexpr int pipe_threads(int cw) { return 32 * (cw + kPipeProducers); }

__device__ __forceinline__ bool tile_interior(const TileInfo& ti, const TileArgs& ta) {
  return ti.cx >= 1 && ti.cx <= ta.n - 2 && ti.cy >= 1 && ti.cy <= ta.n - 2 && ti.z0 >= 1 && ti.z0 + ti.Tp <= ta.n - 1;
}

// FP64 half list, by the producer warp: the sorted indices of a staged tile (the consumers put the
// periodic images in place, as for the mixed form).
__device__ __forceinline__ void stage_gid_warp(const TileShared& S, unsigned char* smem, const TileLayout& L,
                                               int lane) {
  for (int q = 0; q < S.ncell; ++q) {
    const int a = S.offq[q], b = S.offq[q + 1], gq = S.g0[q];
    for (int e = a + lane; e < b; e += 32) ((int*)(smem + L.gid))[e] = gq + (e - a);
  }
}

// Image shifts of a staged tile's periodic cells by the consumer warps (warp per cell, lanes over
// its particles): integer adds of round(L / u) to the fixed-point records.  Every writer orders its
// writes before later bulk copies into the same bytes; the caller then waits for all consumer
// warps (a bounded mbarrier wait, not bar.sync, so that a warp that left on a timeout cannot hold
// the others forever).
template <bool MIXED>
__device__ __forceinline__ void stage_shift_consumers(const TileInfo& ti, const TileArgs& ta, const Geom& g,
                                                      const TileShared& S, unsigned char* smem, const TileLayout& L,
                                                      int consumers) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int q = warp; q < S.ncell; q += consumers) {
    int sx, sy, sz;
    cell_of_q(ti, ta.n, S.ncol, q, sx, sy, sz);
    if ((sx | sy | sz) == 0) continue;
    for (int e = S.offq[q] + lane; e < S.offq[q + 1]; e += 32) {
      if (MIXED) {
        uint4* r = (uint4*)(smem + L.pos) + e;
        r->x = shift_q(r->x, sx, g);
        r->y = shift_q(r->y, sy, g);
        r->z = shift_q(r->z, sz, g);
      } else {  // FP64: s L added, one rounding per staged coordinate instead of a shift per pair
        dvec4* p = (dvec4*)(smem + L.pos) + e;
        p->x += (double)sx * g.L;
        p->y += (double)sy * g.L;
        p->z += (double)sz * g.L;
      }
    }
  }
  fence_proxy_async_smem();
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// CW consumer warps: 8 for tiles of up to 4 cells, 12 for larger tiles (more keys per tile).
// Forms: the mixed form with the full list and the FP64 form with the half list (the producer writes
// the sorted indices; the consumers scatter the partners' forces with atomics).  The consumers put
// the periodic images of a boundary tile in place before computing it.
template <bool MIXED, bool HALF, int LANES, bool ENERGY, bool LONGLIST, int CW>
__global__ void __launch_bounds__(pipe_threads(CW), (MIXED && CW <= 8) ? 3 : 2)
    k_force_pipe(const void* __restrict__ pos, const uint32_t* __restrict__ cs, Geom g, TileArgs ta, LJConst c,
                 const uint2* __restrict__ rows, const uint2* __restrict__ tile_list,
                 const uint16_t* __restrict__ ent, void* __restrict__ fout, double* __restrict__ part,
                 int32_t* __restrict__ status, const int* __restrict__ skip) {
  static_assert(MIXED != HALF, "pipelined forms: mixed with the full list, FP64 with the half list");
  if (skip && *skip) return;  // a device-decided run stopped before this step
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ TileShared SS[kPipeSlots];
  __shared__ TileInfo s_ti[kPipeSlots];
  __shared__ int s_valid[kPipeSlots];  // 1: interior tile, 2: periodic tile (shifts), 0: skip, -1: abort
  __shared__ __align__(8) uint64_t full[2], ready[2], empty[2], shifted[2];
  const TileLayout L = tile_layout(ta, MIXED, true, !MIXED && HALF);
  const size_t buf_bytes = align16(L.total);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&ready[b], 1);
      mbar_init(&empty[b], CW);
      mbar_init(&shifted[b], CW);
    }
    fence_proxy_async_smem();
  }
  __syncthreads();
  EAcc eacc;
  eacc.vscale = g.qu;
  const int64_t stride = gridDim.x;
  if (warp >= CW) {
    // ---- producer p: tiles k = p, p + 2, ... in buffer p ----
    const int p = warp - CW, b = p;
    int64_t t = blockIdx.x + p * stride;
    TilePrefetch pf;
    bool ok_next = false;
    TileInfo ti_cur{0, 0, 0, 0};
    if (t < ta.ntiles) {
      tile_prefetch(t, ta, cs, tile_list, pf, lane);
      ti_cur = pf.ti;
      ok_next = tile_prepare_pf(pf, ta, SS[p], lane);
      if (t + 2 * stride < ta.ntiles) tile_prefetch(t + 2 * stride, ta, cs, tile_list, pf, lane);
    }
    for (int k = p; t < ta.ntiles; t += 2 * stride, k += 2) {
      const int slot = k % kPipeSlots;
      const uint32_t use = (uint32_t)(k >> 1);
      TileShared& S = SS[slot];
      unsigned char* buf = smem + b * buf_bytes;
      bool ok = true;
      if (k >= 2) {
        if (lane == 0) ok = mbar_wait(&empty[b], (use - 1u) & 1u, wait_budget());
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      }
      if (!ok) {  // the consumers did not release the buffer: give up (nothing in flight)
        if (lane == 0) {
          atomicOr(status, LJ_ST_TIMEOUT);
          s_valid[slot] = -1;
          mbar_arrive(&ready[b]);
        }
        break;
      }
      const TileInfo ti = ti_cur;
      bool staged = ok_next;
      if (staged && (S.own1 - S.own0 > ta.max_own || S.list_len > (unsigned)ta.max_list)) {
        if (lane == 0) atomicOr(status, LJ_ST_LIST_OVERFLOW);
        staged = false;
      }
      if (!staged && lane == 0 && !ok_next) atomicOr(status, LJ_ST_CELL_RANGE);
      if (staged) stage_issue<MIXED, true>(ti, ta, pos, rows, ent, S, buf, L, &full[b], warp);
      // bookkeeping of this producer's next tile (its slot was released with tile k - 2), then
      // the loads for the one after it
      const int64_t tn = t + 2 * stride;
      if (tn < ta.ntiles) {
        ti_cur = pf.ti;
        ok_next = tile_prepare_pf(pf, ta, SS[(k + 2) % kPipeSlots], lane);
        if (tn + 2 * stride < ta.ntiles) tile_prefetch(tn + 2 * stride, ta, cs, tile_list, pf, lane);
      }
      if (staged) {
        bool landed = true;
        if (lane == 0) landed = mbar_wait(&full[b], use & 1u, wait_budget());
        landed = __shfl_sync(0xffffffffu, landed ? 1 : 0, 0) != 0;
        if (!landed) {
          if (lane == 0) {
            atomicOr(status, LJ_ST_TIMEOUT);
            mbar_wait(&full[b], use & 1u, kWaitBudget);  // let copies in flight land before leaving
            s_valid[slot] = -1;
            mbar_arrive(&ready[b]);
          }
          break;
        }
        if (!MIXED) {  // sorted indices by this warp; they precede later bulk copies
          stage_gid_warp(S, buf, L, lane);
          fence_proxy_async_smem();
          __syncwarp();
        }
      }
      if (lane == 0) {
        s_ti[slot] = ti;
        s_valid[slot] = staged ? (tile_interior(ti, ta) ? 1 : 2) : 0;
        mbar_arrive(&ready[b]);  // release: bookkeeping and copies visible to the consumers
      }
    }
  } else {
    // ---- consumers ----
    int k = 0;
    uint32_t shpar = 0u;  // bit b: phase of shifted[b] (every consumer warp sees the same tiles)
    for (int64_t t = blockIdx.x; t < ta.ntiles; t += stride, ++k) {
      const int b = k & 1, slot = k % kPipeSlots;
      const uint32_t use = (uint32_t)(k >> 1);
      bool ok = __all_sync(0xffffffffu, mbar_wait(&ready[b], use & 1u, wait_budget())) != 0;
      if (!ok) {
        if (lane == 0) atomicOr(status, LJ_ST_TIMEOUT);
        break;
      }
      const int v = s_valid[slot];
      if (v < 0) break;
      unsigned char* buf = smem + b * buf_bytes;
      if (v == 2) {  // periodic tile: shifts by all consumer warps, then wait for all of them
        stage_shift_consumers<MIXED>(s_ti[slot], ta, g, SS[slot], buf, L, CW);
        __syncwarp();
        if (lane == 0) mbar_arrive(&shifted[b]);
        ok = __all_sync(0xffffffffu, mbar_wait(&shifted[b], (shpar >> b) & 1u, wait_budget())) != 0;
        shpar ^= 1u << b;
        if (!ok) {
          if (lane == 0) atomicOr(status, LJ_ST_TIMEOUT);
          break;
        }
      }
      if (v > 0)
        force_tile_compute<MIXED, LANES, HALF, ENERGY, false, LONGLIST, 32 * CW>(SS[slot], buf, L, rows, ent, c, g,
                                                                                    fout, status, eacc, ta.list_cap);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[b]);
    }
  }
  __syncthreads();
  if (ENERGY) {
    __shared__ double sh[32];
    eacc.flush();
    const double tp = block_sum(eacc.pe, sh);
    __syncthreads();
    const double tv = block_sum(eacc.vir, sh);
    if (threadIdx.x == 0) {
      part[2 * (size_t)blockIdx.x] = tp;
      part[2 * (size_t)blockIdx.x + 1] = tv;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Batched replicas (mixed form, full list): one persistent launch walks the tiles of all
// replicas; each tile takes its replica's box and grid from the replica table.  Energies: the
// tile's PE and virial are reduced over the CTA and added to its replica's totals (e_rep[2 r],
// e_rep[2 r + 1]).
template <int LANES, bool ENERGY>
__global__ void __launch_bounds__(kTileThreads, 4)
    k_force_batch(const uint4* __restrict__ pos, const uint32_t* __restrict__ cs_in, int64_t N, TileArgs caps,
                  LJConst c, const uint2* __restrict__ rows,
                  const uint2* __restrict__ tile_list, const uint16_t* __restrict__ ent, float4* __restrict__ fout,
                  double* __restrict__ e_rep, int32_t* __restrict__ status, const ReplicaGeo* __restrict__ reps,
                  int R, const int32_t* __restrict__ tile_rep) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ TileShared S;
  __shared__ __align__(8) uint64_t bar;
  __shared__ double sh[32];
  const TileLayout L = tile_layout(caps, true, true, false);
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_proxy_async_smem();
  }
  __syncthreads();
  uint32_t ph = 0;
  for (int64_t t = blockIdx.x; t < caps.ntiles; t += gridDim.x) {
    const int r = tile_rep[t];
    const ReplicaGeo& rg = reps[r];
    TileArgs ta = caps;
    Geom g;
    replica_view(rg, ta, g);
    const uint32_t* cs = cs_in + rg.cell_base;
    const TileInfo ti = tile_info(t - rg.tile_base, ta);
    EAcc eacc;
    eacc.vscale = g.qu;
    if (force_tile_prepare(ti, t, ta, cs, tile_list, S, status)) {
      stage_issue<true, true>(ti, ta, pos, rows, ent, S, smem, L, &bar);
      if (!stage_finish<true, true>(ti, ta, g, S, smem, L, &bar, ph, false, status)) return;
      force_tile_compute<true, LANES, false, ENERGY, false, true>(S, smem, L, rows, ent, c, g, fout, status, eacc,
                                                                  ta.list_cap);
    }
    if (ENERGY) {
      eacc.flush();
      const double tp = block_sum(eacc.pe, sh);
      __syncthreads();
      const double tv = block_sum(eacc.vir, sh);
      if (threadIdx.x == 0) {
        atomicAdd(&e_rep[2 * r], 0.5 * tp);  // full list: each pair twice
        atomicAdd(&e_rep[2 * r + 1], 0.5 * tv);
      }
    }
    __syncthreads();
  }
}

// Largest staged and own counts over the tiles of all replicas.
__global__ void k_tile_sizes_batch(const uint32_t* __restrict__ cs_in, TileArgs caps,
                                   const ReplicaGeo* __restrict__ reps, int R, const int32_t* __restrict__ tile_rep,
                                   unsigned int* __restrict__ out) {
  unsigned int mst = 0, mown = 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < caps.ntiles;
       t += (int64_t)gridDim.x * blockDim.x) {
    const ReplicaGeo& rg = reps[tile_rep[t]];
    TileArgs ta = caps;
    Geom g;
    replica_view(rg, ta, g);
    const uint32_t* cs = cs_in + rg.cell_base;
    const TileInfo ti = tile_info(t - rg.tile_base, ta);
    const int ncol = ti.Tp + 2;
    unsigned int tot = 0;
    for (int q = 0; q < 9 * ncol; ++q) {
      int sx, sy, sz;
      const uint32_t cq = cell_of_q(ti, ta.n, ncol, q, sx, sy, sz);
      tot += cs[cq + 1] - cs[cq];
    }
    const uint32_t c0 = ((uint32_t)ti.cx * (uint32_t)ta.n + (uint32_t)ti.cy) * (uint32_t)ta.n + (uint32_t)ti.z0;
    mst = max(mst, tot);
    mown = max(mown, cs[c0 + ti.Tp] - cs[c0]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mst = max(mst, __shfl_xor_sync(0xffffffffu, mst, o));
    mown = max(mown, __shfl_xor_sync(0xffffffffu, mown, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out[0], mst);
    atomicMax(&out[1], mown);
  }
}

// ---------------------------------------------------------------------------------------------
// Adjoint pass over the list (the derivatives the reverse-time recurrences need), for the pair
// energy u(s) of Eq. 2 as a function of s = r^2 (a = sigma^2 / s):
//   u   = 4 eps (a^6 - a^3 + c2 s / sigma^2 + c0)
//   u'  = du/ds   = 4 eps ((3 a^3 - 6 a^6) / s + c2 / sigma^2)
//   u'' = d2u/ds2 = 4 eps (42 a^6 - 12 a^3) / s^2
//   du/dsigma  = (4 eps / sigma) (12 a^6 - 6 a^3 - 2 c2 s / sigma^2)
//   du'/dsigma = (4 eps / sigma) ((18 a^3 - 72 a^6) / s - 2 c2 / sigma^2)
// (c2, c0 fixed: r_c scales with sigma).  Per key i, with d = x_j - x_i and dw = w_i - w_j:
//   (H w)_i += 2 u' dw + 4 u'' d (d . dw)        (Hessian of the potential energy times w)
//   F_i     += 2 u' d                              (force, = -dPE/dx_i)
//   w . dF/dsigma += w_i . (2 du'/dsigma d),  w . dF/deps += w_i . (2 u' d) / eps
//   PE += u / 2,  dPE/deps += u / (2 eps),  dPE/dsigma += (du/dsigma) / 2   (full list: each pair twice)
// all zero for s >= r_c^2.  Block partials: [w.dF/deps, w.dF/dsigma, dPE/deps, dPE/dsigma, PE].
constexpr int kAdjLanes = 4;
constexpr int kAdjParts = 5;

template <bool MIXED, bool WHOLE>
__device__ __forceinline__ void adjoint_tile_compute(const TileShared& S, const unsigned char* buf, const TileLayout& L,
                                                     const uint2* __restrict__ rows, const uint16_t* __restrict__ ent,
                                                     const LJConst& c, const Geom& g, const dvec4* __restrict__ w,
                                                     const float4* __restrict__ wf, dvec4* __restrict__ hw,
                                                     dvec4* __restrict__ fo, int32_t* __restrict__ status, double* acc,
                                                     int list_cap) {
  const void* sh_pos = buf + L.pos;
  const int* sh_gid = (const int*)(buf + L.gid);
  const uint2* s_rows = (const uint2*)(buf + L.rows);
  const uint16_t* s_ent = (const uint16_t*)(buf + L.ent);
  const int lane = threadIdx.x & (kAdjLanes - 1);
  const int grp = threadIdx.x / kAdjLanes;
  constexpr int kGroups = kTileThreads / kAdjLanes;
  const double e4 = 4.0 * c.eps, inv_sig = c.inv_sigma, c2s = c.c2s;
  const int n_own = S.own1 - S.own0;
  for (int o = grp; __any_sync(0xffffffffu, o < n_own); o += kGroups) {
    const bool valid = o < n_own;
    double h[3] = {0.0, 0.0, 0.0}, f[3] = {0.0, 0.0, 0.0}, q[kAdjParts] = {0.0, 0.0, 0.0, 0.0, 0.0};
    float ah[3] = {0.f, 0.f, 0.f}, af[3] = {0.f, 0.f, 0.f}, aq[kAdjParts] = {0.f, 0.f, 0.f, 0.f, 0.f};
    int gi = 0;
    if (valid) {
      const int l = S.own0 + o;
      gi = S.gown0 + o;
      uint2 row;
      const uint16_t* el;
      if (WHOLE) {
        row = rows[gi];
        el = ent;
      } else {
        row = s_rows[S.row_off + o];
        row.x -= S.list_base;
        el = S.list_len <= (unsigned)list_cap ? s_ent : ent + S.list_base;  // long segments stay in HBM
        if (row.x + row.y > S.list_len) {
          if (lane == 0) atomicOr(status, LJ_ST_LIST_OVERFLOW);
          row.y = 0;
        }
      }
      if (MIXED) {
        const uint4 qi = ((const uint4*)sh_pos)[l];
        const float e4f = c.e4, sig2f = c.sig2f, c2sf = c.c2sf, rc2f = c.rc2f, c0f = c.c0f, isgf = c.inv_sigmaf;
        const float4 wif = wf[gi];  // the FP32 copy of w (no conversions per pair)
        const float wx = wif.x, wy = wif.y, wz = wif.z;
        for (unsigned e = lane; e < row.y; e += kAdjLanes) {
          const int j = el[row.x + e];
          const uint4 qj = ((const uint4*)sh_pos)[j];
          // differences in sigma units: the integer difference in units of u, converted once and
          // scaled by u (a power of two: exact)
          const float dx = qd<WHOLE>(qj.x, qi.x, g) * g.qu, dy = qd<WHOLE>(qj.y, qi.y, g) * g.qu,
                      dz = qd<WHOLE>(qj.z, qi.z, g) * g.qu;
          const float s2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          if (!(s2 < rc2f)) continue;
          const float4 wj = wf[qj.w];
          const float is = rcp_nr(s2);
          const float a = sig2f * is, a3 = a * a * a, a6 = a3 * a3;
          const float u = e4f * (a6 - a3 + c2sf * s2 + c0f);
          const float u1 = e4f * (is * (3.0f * a3 - 6.0f * a6) + c2sf);
          const float u2 = e4f * is * is * (42.0f * a6 - 12.0f * a3);
          const float dus = e4f * isgf * (12.0f * a6 - 6.0f * a3 - 2.0f * c2sf * s2);
          const float du1s = e4f * isgf * (is * (18.0f * a3 - 72.0f * a6) - 2.0f * c2sf);
          const float dwx = wx - wj.x, dwy = wy - wj.y, dwz = wz - wj.z;
          const float ddw = dx * dwx + dy * dwy + dz * dwz;
          const float t1 = 2.0f * u1, t2 = 4.0f * u2 * ddw;
          ah[0] += t1 * dwx + t2 * dx;
          ah[1] += t1 * dwy + t2 * dy;
          ah[2] += t1 * dwz + t2 * dz;
          af[0] += t1 * dx;
          af[1] += t1 * dy;
          af[2] += t1 * dz;
          const float wd = wx * dx + wy * dy + wz * dz;
          aq[0] += t1 * wd;
          aq[1] += 2.0f * du1s * wd;
          aq[2] += 0.5f * u;
          aq[3] += 0.5f * dus;
          aq[4] += 0.5f * u;
        }
      } else {
        const dvec4 wi = w[gi];
        const dvec4 qi = ((const dvec4*)sh_pos)[l];
        for (unsigned e = lane; e < row.y; e += kAdjLanes) {
          const int j = el[row.x + e];
          const dvec4 qj = ((const dvec4*)sh_pos)[j];  // its image already in place (tiles)
          double dx = qj.x - qi.x, dy = qj.y - qi.y, dz = qj.z - qi.z;
          if (WHOLE) {
            dx = fma(-rint(dx * g.inv_L64), g.L, dx);
            dy = fma(-rint(dy * g.inv_L64), g.L, dy);
            dz = fma(-rint(dz * g.inv_L64), g.L, dz);
          }
          const double s2 = fma(dx, dx, fma(dy, dy, dz * dz));
          if (!(s2 < c.rc2)) continue;
          const dvec4 wj = w[sh_gid[j]];
          const double is = rcp_nr64(s2);
          const double a = c.sig2 * is, a3 = a * a * a, a6 = a3 * a3;
          const double u = e4 * (a6 - a3 + c2s * s2 + c.c0);
          const double u1 = e4 * (is * (3.0 * a3 - 6.0 * a6) + c2s);
          const double u2 = e4 * is * is * (42.0 * a6 - 12.0 * a3);
          const double dus = e4 * inv_sig * (12.0 * a6 - 6.0 * a3 - 2.0 * c2s * s2);
          const double du1s = e4 * inv_sig * (is * (18.0 * a3 - 72.0 * a6) - 2.0 * c2s);
          const double dwx = wi.x - wj.x, dwy = wi.y - wj.y, dwz = wi.z - wj.z;
          const double ddw = dx * dwx + dy * dwy + dz * dwz;
          const double t1 = 2.0 * u1, t2 = 4.0 * u2 * ddw;
          h[0] += t1 * dwx + t2 * dx;
          h[1] += t1 * dwy + t2 * dy;
          h[2] += t1 * dwz + t2 * dz;
          f[0] += t1 * dx;
          f[1] += t1 * dy;
          f[2] += t1 * dz;
          const double wd = wi.x * dx + wi.y * dy + wi.z * dz;
          q[0] += t1 * wd;
          q[1] += 2.0 * du1s * wd;
          q[2] += 0.5 * u;
          q[3] += 0.5 * dus;
          q[4] += 0.5 * u;
        }
      }
    }
    if (MIXED) {  // the group's lanes reduce in FP32; one lane converts and accumulates in FP64
      for (int k = 0; k < 3; ++k) {
        ah[k] = gsum<kAdjLanes>(ah[k]);
        af[k] = gsum<kAdjLanes>(af[k]);
      }
      for (int k = 0; k < kAdjParts; ++k) aq[k] = gsum<kAdjLanes>(aq[k]);
      if (valid && lane == 0) {
        hw[gi] = make_dvec4(ah[0], ah[1], ah[2], 0.0);
        if (fo) fo[gi] = make_dvec4(af[0], af[1], af[2], 0.0);
        for (int k = 0; k < kAdjParts; ++k) acc[k] += (double)aq[k];
      }
    } else {
      for (int k = 0; k < 3; ++k) {
        h[k] = gsum<kAdjLanes>(h[k]);
        f[k] = gsum<kAdjLanes>(f[k]);
      }
      if (valid && lane == 0) {
        hw[gi] = make_dvec4(h[0], h[1], h[2], 0.0);
        if (fo) fo[gi] = make_dvec4(f[0], f[1], f[2], 0.0);
      }
      for (int k = 0; k < kAdjParts; ++k) acc[k] += q[k];
    }
  }
}

template <bool MIXED, bool WHOLE>
__global__ void __launch_bounds__(kTileThreads, 2)
    k_adjoint_tile(const void* __restrict__ pos, const uint32_t* __restrict__ cs, int64_t N, Geom g, TileArgs ta,
                   LJConst c, const uint2* __restrict__ rows,
                   const uint2* __restrict__ tile_list, const uint16_t* __restrict__ ent,
                   const dvec4* __restrict__ w, const float4* __restrict__ wf, dvec4* __restrict__ hw,
                   dvec4* __restrict__ fo, double* __restrict__ part, unsigned int* __restrict__ ticket,
                   double* __restrict__ sums, int32_t* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ TileShared S;
  __shared__ __align__(8) uint64_t bar;
  const TileLayout L = tile_layout(ta, MIXED, true, !MIXED);
  double acc[kAdjParts] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (WHOLE) {
    if (blockIdx.x == 0) {
      stage_whole<MIXED, !MIXED>(N, pos, S, smem, L);
      __syncthreads();
      adjoint_tile_compute<MIXED, true>(S, smem, L, rows, ent, c, g, w, wf, hw, fo, status, acc, ta.list_cap);
    }
  } else {
    if (threadIdx.x == 0) {
      mbar_init(&bar, 1);
      fence_proxy_async_smem();
    }
    __syncthreads();
    uint32_t ph = 0;
    for (int64_t t = blockIdx.x; t < ta.ntiles; t += gridDim.x) {
      const bool ok = force_tile_prepare(tile_info(t, ta), t, ta, cs, tile_list, S, status);
      if (ok) {
        const TileInfo ti = tile_info(t, ta);
        stage_issue<MIXED, true>(ti, ta, pos, rows, ent, S, smem, L, &bar);
        if (!stage_finish<MIXED, true>(ti, ta, g, S, smem, L, &bar, ph, !MIXED, status)) return;
        adjoint_tile_compute<MIXED, false>(S, smem, L, rows, ent, c, g, w, wf, hw, fo, status, acc, ta.list_cap);
      }
      __syncthreads();
    }
  }
  __shared__ double sh[32];
  for (int k = 0; k < kAdjParts; ++k) {
    const double t = block_sum(acc[k], sh);
    if (threadIdx.x == 0) part[kAdjParts * (size_t)blockIdx.x + k] = t;
    __syncthreads();
  }
  // the last CTA to finish sums the partials of all CTAs in block order (thread 0 wrote this CTA's
  // partials and orders them before its ticket)
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    for (int k = 0; k < kAdjParts; ++k) {
      double v = 0.0;
      for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) v += __ldcg(part + kAdjParts * (size_t)b + k);
      v = block_sum(v, sh);
      if (threadIdx.x == 0) sums[k] = v;
      __syncthreads();
    }
    if (threadIdx.x == 0) *ticket = 0u;
  }
}


// ---------------------------------------------------------------------------------------------
// Expand the list into (key, partner) sorted-index pairs (for inspection).  The whole-box case
// is a template parameter: no barrier sits under a runtime branch.
template <bool WHOLE>
__global__ void __launch_bounds__(kTileThreads, 4)
    k_list_decode(const uint32_t* __restrict__ cs, int64_t N, TileArgs ta, const uint2* __restrict__ rows,
                  const uint16_t* __restrict__ ent, uint64_t E, uint32_t* __restrict__ out,
                  int32_t* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ TileShared S;
  int* sh_gid = (int*)smem;
  for (int64_t t = blockIdx.x; t < ta.ntiles; t += gridDim.x) {
    if (WHOLE) {
      for (int e = threadIdx.x; e < N; e += blockDim.x) sh_gid[e] = e;
      if (threadIdx.x == 0) {
        S.own0 = 0;
        S.own1 = (int)N;
        S.total = (int)N;
      }
    } else {
      const TileInfo ti = tile_info(t, ta);
      if (!stage_offsets(ti, ta, cs, S)) {
        if (threadIdx.x == 0) atomicOr(status, LJ_ST_CELL_RANGE);
        __syncthreads();
        continue;
      }
      for (int s = threadIdx.x; s < S.total; s += blockDim.x) {
        const int q = slot_cell(S, s);
        sh_gid[s] = S.g0[q] + (s - S.offq[q]);
      }
    }
    __syncthreads();
    for (int l = S.own0 + (int)threadIdx.x / 32; l < S.own1; l += kWarps) {
      const int gi = sh_gid[l];
      const uint2 row = rows[gi];
      if ((uint64_t)row.x + row.y > E) {  // inconsistent row: record and skip
        if ((threadIdx.x & 31) == 0) atomicOr(status, LJ_ST_LIST_OVERFLOW);
        continue;
      }
      for (unsigned e = threadIdx.x & 31; e < row.y; e += 32) {
        const int j = ent[row.x + e];
        const bool ok = j < S.total;
        if (!ok) atomicOr(status, LJ_ST_LIST_OVERFLOW);
        out[2 * (size_t)(row.x + e)] = (uint32_t)gi;
        out[2 * (size_t)(row.x + e) + 1] = ok ? (uint32_t)sh_gid[j] : 0xffffffffu;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// Sets the budget of the bounded device waits (0: the default).  Synchronises the device.
int set_wait_budget(long long cycles) {
  const long long v = cycles > 0 ? cycles : kWaitBudget;
  if (cudaDeviceSynchronize() != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(g_wait_budget, &v, sizeof(v)) != cudaSuccess) return -1;
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : -1;
}

static int sm_count() {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

static int tile_grid(const TileArgs& ta, int per_sm) {
  int64_t b = (int64_t)sm_count() * per_sm;
  if (b > ta.ntiles) b = ta.ntiles;
  if (b > kMaxRedBlocks) b = kMaxRedBlocks;
  return (int)(b < 1 ? 1 : b);
}

template <class K>
static void set_smem(K kernel, size_t bytes) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// CTAs of a kernel resident per SM at the given dynamic shared memory (registers included).
template <class K>
static int resident_per_sm(K kernel, int threads, size_t smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess || nb < 1) nb = 1;
  return nb;
}

static int per_sm_for(size_t smem_bytes) {
  int dev = 0, smem_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  int k = (int)(smem_sm / (int)(smem_bytes + sizeof(TileShared) + 1024));
  return k < 1 ? 1 : (k > 4 ? 4 : k);
}

void launch_list_tile(int precision, int half, const void* pos, const float4* hi, const double* x, const uint32_t* cs,
                      int64_t N, Geom g, TileArgs ta, ListBand band, uint2* rows, uint2* tile_list, uint16_t* ent,
                      uint64_t cap, unsigned long long* counter, unsigned int* max_list, int32_t* status,
                      cudaStream_t s) {
  const size_t sm = list_smem_bytes(ta, precision);
  int grid = tile_grid(ta, per_sm_for(sm));
  if (!ta.whole) {  // the window kernel: as many CTAs as are resident
    set_smem(k_list_win<false, false, kWinThreads>, sm);
    grid = tile_grid(ta, resident_per_sm(k_list_win<false, false, kWinThreads>, kWinThreads, sm));
  }
#define LJ_LIST_LAUNCH(M, H, W)                                                                                 \
  do {                                                                                                          \
    set_smem(k_list_tile<M, H, W>, sm);                                                                         \
    k_list_tile<M, H, W><<<grid, kTileThreads, sm, s>>>(pos, x, cs, N, g, ta, band, rows, tile_list, ent, cap, \
                                                        counter, max_list, status);                             \
  } while (0)
  const bool mixed = precision == LJ_MIXED;
  if (ta.whole) {
    if (mixed) {
      if (half) LJ_LIST_LAUNCH(true, true, true);
      else LJ_LIST_LAUNCH(true, false, true);
    } else {
      if (half) LJ_LIST_LAUNCH(false, true, true);
      else LJ_LIST_LAUNCH(false, false, true);
    }
  } else if (half) {  // tiles, either form: one thread per key on the hi copies (the list is the same)
    set_smem(k_list_win<true, false, kWinThreads>, sm);
    k_list_win<true, false, kWinThreads><<<grid, kWinThreads, sm, s>>>(hi, x, cs, N, g, ta, band, rows, tile_list, ent,
                                                                       cap, counter, max_list, status, nullptr, 0,
                                                                       nullptr, nullptr);
  } else {
    set_smem(k_list_win<false, false, kWinThreads>, sm);
    k_list_win<false, false, kWinThreads><<<grid, kWinThreads, sm, s>>>(hi, x, cs, N, g, ta, band, rows, tile_list, ent,
                                                                        cap, counter, max_list, status, nullptr, 0,
                                                                        nullptr, nullptr);
  }
#undef LJ_LIST_LAUNCH
}

// Returns the grid launched (the number of energy partials written).
template <bool MIXED, int LANES, bool HALF, bool ENERGY>
static int force_w(const void* pos, const uint32_t* cs, int64_t N, Geom g, TileArgs ta, LJConst c, const uint2* rows,
                   const uint2* tl, const uint16_t* ent, void* f, double* part, int32_t* status, int nbuf, int grid,
                   size_t sm, cudaStream_t s, const int* skip) {
#define LJ_FW(W, LONG)                                                                                           \
  do {                                                                                                           \
    set_smem(k_force_tile<MIXED, LANES, HALF, ENERGY, W, LONG>, sm);                                             \
    k_force_tile<MIXED, LANES, HALF, ENERGY, W, LONG><<<grid, kTileThreads, sm, s>>>(pos, cs, N, g, ta, c, rows,   \
                                                                                    tl, ent, f, part, status, nbuf,  \
                                                                                    skip);                          \
  } while (0)
  if constexpr (MIXED != HALF) {  // the pipelined forms: mixed + full list, FP64 + half list
    if (!ta.whole && nbuf == 2) {  // producer warps + consumer warps over two buffers
#define LJ_FP(LONG, CW)                                                                                          \
  do {                                                                                                           \
    set_smem(k_force_pipe<MIXED, HALF, LANES, ENERGY, LONG, CW>, sm);                                            \
    const int64_t want = (int64_t)sm_count() *                                                                   \
                         resident_per_sm(k_force_pipe<MIXED, HALF, LANES, ENERGY, LONG, CW>, pipe_threads(CW), sm); \
    grid = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(want, ta.ntiles), (int64_t)kMaxRedBlocks)); \
    k_force_pipe<MIXED, HALF, LANES, ENERGY, LONG, CW><<<grid, pipe_threads(CW), sm, s>>>(pos, cs, g, ta, c, rows, \
                                                                                       tl, ent, f, part, status,      \
                                                                                       skip);                         \
  } while (0)
      const bool lg = ta.list_cap < ta.max_list;
      if (ta.T <= 4) {
        if (lg) LJ_FP(true, 8);
        else LJ_FP(false, 8);
      } else {
        if (lg) LJ_FP(true, 12);
        else LJ_FP(false, 12);
      }
#undef LJ_FP
      return grid;
    }
  }
  if (ta.whole) LJ_FW(true, false);
  else if (ta.list_cap < ta.max_list) LJ_FW(false, true);  // some segments longer than the staged capacity
  else LJ_FW(false, false);
#undef LJ_FW
  return grid;
}

template <bool MIXED, int LANES>
static int force_l(int half, int energy, const void* pos, const uint32_t* cs, int64_t N, Geom g, TileArgs ta,
                   LJConst c, const uint2* rows, const uint2* tl, const uint16_t* ent, void* f, double* part,
                   int32_t* status, int nbuf, int grid, size_t sm, cudaStream_t s, const int* skip) {
  if (half) {
    if (energy) return force_w<MIXED, LANES, true, true>(pos, cs, N, g, ta, c, rows, tl, ent, f, part, status, nbuf, grid, sm, s, skip);
    return force_w<MIXED, LANES, true, false>(pos, cs, N, g, ta, c, rows, tl, ent, f, part, status, nbuf, grid, sm, s, skip);
  }
  if (energy) return force_w<MIXED, LANES, false, true>(pos, cs, N, g, ta, c, rows, tl, ent, f, part, status, nbuf, grid, sm, s, skip);
  return force_w<MIXED, LANES, false, false>(pos, cs, N, g, ta, c, rows, tl, ent, f, part, status, nbuf, grid, sm, s, skip);
}

template <bool MIXED>
static int force_p(int lanes, int half, int energy, const void* pos, const uint32_t* cs, int64_t N, Geom g,
                   TileArgs ta, LJConst c, const uint2* rows, const uint2* tl, const uint16_t* ent, void* f,
                   double* part, int32_t* status, int nbuf, int grid, size_t sm, cudaStream_t s, const int* skip) {
  switch (lanes) {
    case 1: return force_l<MIXED, 1>(half, energy, pos, cs, N, g, ta, c, rows, tl, ent, f, part, status, nbuf, grid, sm, s, skip);
    case 2: return force_l<MIXED, 2>(half, energy, pos, cs, N, g, ta, c, rows, tl, ent, f, part, status, nbuf, grid, sm, s, skip);
    case 4: return force_l<MIXED, 4>(half, energy, pos, cs, N, g, ta, c, rows, tl, ent, f, part, status, nbuf, grid, sm, s, skip);
    case 8: return force_l<MIXED, 8>(half, energy, pos, cs, N, g, ta, c, rows, tl, ent, f, part, status, nbuf, grid, sm, s, skip);
    case 16: return force_l<MIXED, 16>(half, energy, pos, cs, N, g, ta, c, rows, tl, ent, f, part, status, nbuf, grid, sm, s, skip);
    default: return force_l<MIXED, 32>(half, energy, pos, cs, N, g, ta, c, rows, tl, ent, f, part, status, nbuf, grid, sm, s, skip);
  }
}

int launch_force_tile(int precision, int half, int lanes, int energy, const void* pos, const uint32_t* cs, int64_t N,
                      Geom g, TileArgs ta, LJConst c, const uint2* rows, const uint2* tile_list, const uint16_t* ent,
                      void* f, double* part, int32_t* status, int per_sm, int nbuf, cudaStream_t s, const int* skip) {
  const size_t sm = force_smem_bytes(ta, precision, nbuf, half);
  if (per_sm <= 0) per_sm = per_sm_for(sm);
  const int grid = tile_grid(ta, per_sm);
  if (precision == LJ_MIXED)
    return force_p<true>(lanes, half, energy, pos, cs, N, g, ta, c, rows, tile_list, ent, f, part, status, nbuf, grid,
                         sm, s, skip);
  return force_p<false>(lanes, half, energy, pos, cs, N, g, ta, c, rows, tile_list, ent, f, part, status, nbuf, grid,
                        sm, s, skip);
}

void launch_list_decode(const uint32_t* cs, int64_t N, TileArgs ta, const uint2* rows, const uint16_t* ent,
                        uint64_t E, uint32_t* out, int32_t* status, cudaStream_t s) {
  const size_t sm = ((4 * (size_t)ta.max_staged) + 15) & ~(size_t)15;
  const int grid = tile_grid(ta, 4);
  if (ta.whole) {
    set_smem(k_list_decode<true>, sm);
    k_list_decode<true><<<grid, kTileThreads, sm, s>>>(cs, N, ta, rows, ent, E, out, status);
  } else {
    set_smem(k_list_decode<false>, sm);
    k_list_decode<false><<<grid, kTileThreads, sm, s>>>(cs, N, ta, rows, ent, E, out, status);
  }
}

// Largest staged count and own count over all tiles (sizes the shared-memory tiles).
__global__ void k_tile_sizes(const uint32_t* __restrict__ cs, TileArgs ta, unsigned int* __restrict__ out) {
  unsigned int mst = 0, mown = 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ta.ntiles;
       t += (int64_t)gridDim.x * blockDim.x) {
    const TileInfo ti = tile_info(t, ta);
    const int ncol = ti.Tp + 2;
    unsigned int tot = 0;
    for (int q = 0; q < 9 * ncol; ++q) {
      int sx, sy, sz;
      const uint32_t cq = cell_of_q(ti, ta.n, ncol, q, sx, sy, sz);
      tot += cs[cq + 1] - cs[cq];
    }
    const uint32_t c0 = ((uint32_t)ti.cx * (uint32_t)ta.n + (uint32_t)ti.cy) * (uint32_t)ta.n + (uint32_t)ti.z0;
    mst = max(mst, tot);
    mown = max(mown, cs[c0 + ti.Tp] - cs[c0]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mst = max(mst, __shfl_xor_sync(0xffffffffu, mst, o));
    mown = max(mown, __shfl_xor_sync(0xffffffffu, mown, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out[0], mst);
    atomicMax(&out[1], mown);
  }
}

void launch_tile_sizes(const uint32_t* cs, TileArgs ta, unsigned int* out, cudaStream_t s) {
  int64_t b = (ta.ntiles + 255) / 256;
  if (b < 1) b = 1;
  if (b > 4096) b = 4096;
  k_tile_sizes<<<(int)b, 256, 0, s>>>(cs, ta, out);
}

// Largest cell occupancy.
__global__ void k_max_count(const uint32_t* __restrict__ cnt, int64_t n, unsigned int* __restrict__ out) {
  unsigned int m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, cnt[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

void launch_max_count(const uint32_t* cnt, int64_t n, unsigned int* out, cudaStream_t s) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 4096) b = 4096;
  k_max_count<<<(int)b, 256, 0, s>>>(cnt, n, out);
}

size_t adjoint_smem_bytes(const TileArgs& ta, int precision) {
  return align16(tile_layout(ta, precision == LJ_MIXED, true, precision != LJ_MIXED).total);
}

int launch_adjoint_tile(int precision, const void* pos, const uint32_t* cs, int64_t N, Geom g, TileArgs ta, LJConst c,
                        const uint2* rows, const uint2* tile_list, const uint16_t* ent, const void* w,
                        const float4* wf, void* hw, void* fo, double* part, unsigned int* ticket, double* sums,
                        int32_t* status, cudaStream_t s) {
  const size_t sm = adjoint_smem_bytes(ta, precision);
  const int grid = tile_grid(ta, min(per_sm_for(sm), 2));
#define LJ_ADJ_LAUNCH(M, W)                                                                                 \
  do {                                                                                                      \
    set_smem(k_adjoint_tile<M, W>, sm);                                                                     \
    k_adjoint_tile<M, W><<<grid, kTileThreads, sm, s>>>(pos, cs, N, g, ta, c, rows, tile_list, ent,         \
                                                        (const dvec4*)w, wf, (dvec4*)hw, (dvec4*)fo, part,      \
                                                        ticket, sums, status);                                  \
  } while (0)
  if (precision == LJ_MIXED) {
    if (ta.whole) LJ_ADJ_LAUNCH(true, true);
    else LJ_ADJ_LAUNCH(true, false);
  } else {
    if (ta.whole) LJ_ADJ_LAUNCH(false, true);
    else LJ_ADJ_LAUNCH(false, false);
  }
#undef LJ_ADJ_LAUNCH
  return grid;
}


// ---- batched replicas -----------------------------------------------------------------------
size_t batch_list_smem_bytes(const TileArgs& caps) { return win_layout(caps).total; }
size_t batch_force_smem_bytes(const TileArgs& caps) { return align16(tile_layout(caps, true, true, false).total); }

void launch_tile_sizes_batch(const uint32_t* cs, TileArgs caps, const ReplicaGeo* reps, int R,
                             const int32_t* tile_rep, unsigned int* out, cudaStream_t s) {
  int64_t b = (caps.ntiles + 255) / 256;
  if (b < 1) b = 1;
  if (b > 4096) b = 4096;
  k_tile_sizes_batch<<<(int)b, 256, 0, s>>>(cs, caps, reps, R, tile_rep, out);
}

void launch_list_batch(const float4* hi, const double* x, const uint32_t* cs, int64_t N, Geom g, TileArgs caps,
                       ListBand band, uint2* rows, uint2* tile_list, uint16_t* ent, uint64_t cap,
                       unsigned long long* counter, unsigned int* max_list, int32_t* status, const ReplicaGeo* reps,
                       int R, const int32_t* tile_rep, const int* pred, cudaStream_t s) {
  const size_t sm = win_layout(caps).total;
  set_smem(k_list_win<false, true, kWinThreads>, sm);
  const int grid = tile_grid(caps, resident_per_sm(k_list_win<false, true, kWinThreads>, kWinThreads, sm));
  k_list_win<false, true, kWinThreads><<<grid, kWinThreads, sm, s>>>(hi, x, cs, N, g, caps, band, rows, tile_list, ent,
                                                                     cap, counter, max_list, status, reps, R, pred,
                                                                     tile_rep);
}

int launch_force_batch(int lanes, int energy, const uint4* xq, const uint32_t* cs, int64_t N,
                       TileArgs caps, LJConst c, const uint2* rows, const uint2* tile_list, const uint16_t* ent,
                       float4* f, double* e_rep, int32_t* status, const ReplicaGeo* reps, int R,
                       const int32_t* tile_rep, cudaStream_t s) {
  const size_t sm = batch_force_smem_bytes(caps);
  const int grid = tile_grid(caps, per_sm_for(sm));
#define LJ_FB(LN)                                                                                               \
  do {                                                                                                          \
    if (energy) {                                                                                               \
      set_smem(k_force_batch<LN, true>, sm);                                                                    \
      k_force_batch<LN, true><<<grid, kTileThreads, sm, s>>>(xq, cs, N, caps, c, rows, tile_list, ent, f,       \
                                                             e_rep, status, reps, R, tile_rep);                          \
    } else {                                                                                                    \
      set_smem(k_force_batch<LN, false>, sm);                                                                   \
      k_force_batch<LN, false><<<grid, kTileThreads, sm, s>>>(xq, cs, N, caps, c, rows, tile_list, ent, f,      \
                                                              e_rep, status, reps, R, tile_rep);                         \
    }                                                                                                           \
  } while (0)
  switch (lanes) {
    case 2: LJ_FB(2); break;
    case 8: LJ_FB(8); break;
    default: LJ_FB(4); break;
  }
#undef LJ_FB
  return grid;
}


// ---- list validity: the large displacement check (LDC) of Alg. 2 -----------------------------
// L_D = { i : |x_i - x_ref_i| > th } with th = margin - (an upper bound of the largest
// displacement); x_ref are the FP64 positions the list was built from.  Indices beyond `cap` are
// counted but not stored.
__global__ void k_ldc_collect(const double* __restrict__ x, const double* __restrict__ xref, int64_t N, double th2,
                              int32_t* __restrict__ list, unsigned int cap, unsigned int* __restrict__ count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double dx = x[i] - xref[i], dy = x[N + i] - xref[N + i], dz = x[2 * N + i] - xref[2 * N + i];
    if (dx * dx + dy * dy + dz * dz > th2) {
      const unsigned int k = atomicAdd(count, 1u);
      if (k < cap) list[k] = (int32_t)i;
    }
  }
}

// Every pair of L_D: unlisted (the list's own exact FP64 test on the build positions says r >= r_s)
// and now closer than r_c (FP64, with a relative safety of 1e-6) raises *flag.  Block (x, y) takes
// the 16 members 16 x .. 16 x + 15 against the 256 members 256 y + threadIdx.x; pairs a < b only.
constexpr int kLdcRows = 16;
__global__ void __launch_bounds__(256) k_ldc_pairs(const double* __restrict__ x, const double* __restrict__ xref,
                                                   int64_t N, Geom g, const int32_t* __restrict__ list, int m,
                                                   double rs2, double rc2, int* __restrict__ flag) {
  __shared__ double sa[kLdcRows][3];
  __shared__ int ia[kLdcRows];
  const int a0 = blockIdx.x * kLdcRows;
  if (threadIdx.x < kLdcRows) {
    const int a = a0 + threadIdx.x;
    const int i = a < m ? list[a] : 0;
    ia[threadIdx.x] = i;
    for (int k = 0; k < 3; ++k) sa[threadIdx.x][k] = x[k * N + i];
  }
  __syncthreads();
  const int b = blockIdx.y * blockDim.x + threadIdx.x;
  if (b >= m || b <= a0) return;  // some a < b remains only if b > a0
  const int j = list[b];
  const double xj = x[j], yj = x[N + j], zj = x[2 * N + j];
  bool hit = false;
  for (int r = 0; r < kLdcRows; ++r) {
    const int a = a0 + r;
    if (a >= m || a >= b) break;
    double t[3] = {xj - sa[r][0], yj - sa[r][1], zj - sa[r][2]};
    double d2 = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (t[k] > g.half_L) t[k] -= g.L;
      else if (t[k] < -g.half_L) t[k] += g.L;
      d2 += t[k] * t[k];
    }
    if (d2 < rc2 * (1.0 + 1e-6) && !pair_in_exact(xref, N, ia[r], j, g, rs2)) hit = true;
  }
  if (hit) atomicOr(flag, 1);
}

void launch_ldc_collect(const double* x, const double* xref, int64_t N, double th2, int32_t* list, unsigned int cap,
                        unsigned int* count, cudaStream_t s) {
  int64_t b = (N + 255) / 256;
  if (b < 1) b = 1;
  if (b > 65535) b = 65535;
  k_ldc_collect<<<(int)b, 256, 0, s>>>(x, xref, N, th2, list, cap, count);
}
void launch_ldc_pairs(const double* x, const double* xref, int64_t N, Geom g, const int32_t* list, int m, double rs2,
                      double rc2, int* flag, cudaStream_t s) {
  dim3 grid((unsigned)((m + kLdcRows - 1) / kLdcRows), (unsigned)((m + 255) / 256));
  k_ldc_pairs<<<grid, 256, 0, s>>>(x, xref, N, g, list, m, rs2, rc2, flag);
}
}  // namespace ljmd
