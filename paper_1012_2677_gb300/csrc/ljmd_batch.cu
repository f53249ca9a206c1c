// C ABI of the batched-replica path (declared in include/ljmd.h): many independent LJ systems of
// uneven size, density and temperature advanced together.  Every phase is one launch over all
// replicas (the replica of a tile or a particle comes from a table), the rebuild decision stays
// on the device (a flag that the rebuild kernels read), and K steps can be captured once as a CUDA
// graph and replayed.  This file only sizes buffers, records launches and reads back scalars.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ljmd_internal.h"

using namespace ljmd;

struct ljmd_batch {
  int device = 0;
  cudaStream_t st = nullptr;       // the batch's own stream (capturable)
  cudaStream_t user_st = nullptr;  // the caller's stream: every call first waits for its work
  cudaEvent_t user_ev = nullptr;
  ljmd_params prm{};
  bool broken = false;
  int R = 0;
  int64_t N = 0;
  std::vector<int64_t> count, base;
  std::vector<double> box;
  double offset = 0.0, rs = 0.0, disp_limit = 0.0;
  int pw = 0;
  LJConst c{};
  ListBand band{};
  Geom g0{};  // the batch's common offset / p (box fields of replica 0)
  std::vector<ReplicaGeo> reps_h;
  ReplicaGeo* reps = nullptr;
  int32_t* tile_rep = nullptr;  // replica of every global tile
  TileArgs caps{};
  int64_t ncells = 0;
  int tile_T = 4;  // preferred cells per tile along z
  int lanes = 4;   // threads per key in the force kernel
  // device state (sorted by cell within each replica)
  double *x = nullptr, *v = nullptr, *x_alt = nullptr, *v_alt = nullptr;
  float4 *f = nullptr, *hi = nullptr;  // forces; FP32 hi parts of the positions (list filter)
  uint4 *xq = nullptr, *ref = nullptr;  // fixed-point position records (force); the records at the build
  int32_t *id = nullptr, *id_alt = nullptr, *img = nullptr, *img_alt = nullptr, *rep_of = nullptr;
  uint32_t *cell_of = nullptr, *perm = nullptr, *perm_id = nullptr, *cell_count = nullptr, *cell_start = nullptr, *cell_fill = nullptr;
  uint32_t* scan_tmp = nullptr;
  uint2 *rows = nullptr, *tile_list = nullptr;
  uint16_t* ent = nullptr;
  size_t ent_cap = 0;
  double *e_rep = nullptr, *ke_rep = nullptr;
  int32_t* status = nullptr;
  uint32_t* dmax = nullptr;
  int* flag = nullptr;
  long long* d_rebuilds = nullptr;
  unsigned long long* counter = nullptr;
  unsigned int* sizes = nullptr;
  // bookkeeping
  bool have_state = false, have_list = false, forces_current = false;
  int64_t steps = 0, host_rebuilds = 0;
  uint64_t list_entries = 0, list_actual = 0;
  int64_t launches = 0;
  // captured K-step graph
  cudaGraphExec_t gexec = nullptr;
  int64_t g_steps = 0;
  double g_dt = 0.0;
  int64_t g_launches = 0;  // kernels per replay
  // pinned host mirrors
  double* h_f64 = nullptr;
  unsigned long long* h_u64 = nullptr;
};

#define BK(call)                     \
  do {                               \
    cudaError_t e_ = (call);         \
    if (e_ != cudaSuccess) {         \
      b->broken = true;              \
      return LJ_EDEVICE;             \
    }                                \
  } while (0)
#define BKL() BK(cudaGetLastError())
#define BTRY(expr)               \
  do {                           \
    int r_ = (expr);             \
    if (r_ != LJ_OK) return r_;  \
  } while (0)

template <class T>
static int balloc(T** p, size_t count) {
  if (*p) cudaFree(*p);
  *p = nullptr;
  if (cudaMalloc((void**)p, (count ? count : 1) * sizeof(T)) != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return LJ_ENOMEM;
  }
  return LJ_OK;
}

static void drop_graph(ljmd_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  b->g_steps = 0;
}

static void free_batch(ljmd_batch* b) {
  drop_graph(b);
  void* ptrs[] = {b->reps, b->tile_rep, b->x, b->v, b->x_alt, b->v_alt, b->f, b->hi, b->xq, b->ref, b->id, b->id_alt, b->img,
                  b->img_alt, b->rep_of, b->cell_of, b->perm, b->perm_id, b->cell_count, b->cell_start, b->cell_fill,
                  b->scan_tmp, b->rows, b->tile_list, b->ent, b->e_rep, b->ke_rep, b->status, b->dmax, b->flag,
                  b->d_rebuilds, b->counter, b->sizes};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (b->h_f64) cudaFreeHost(b->h_f64);
  if (b->h_u64) cudaFreeHost(b->h_u64);
  if (b->user_ev) cudaEventDestroy(b->user_ev);
  if (b->st) cudaStreamDestroy(b->st);
}

// Order the batch's stream after the work the caller has queued on its stream so far.
static int join_user(ljmd_batch* b) {
  BK(cudaEventRecord(b->user_ev, b->user_st));
  BK(cudaStreamWaitEvent(b->st, b->user_ev, 0));
  return LJ_OK;
}

// Cells per tile along z for one replica: the preferred T at density 0.5, scaled by 0.5 / rho so that
// a tile stages about the same number of particles in every replica (the shared-memory capacity is
// set by the densest replica's tiles).
static int replica_tile(int pref, int64_t n_cells, int64_t count, double L) {
  const double rho = (double)count / (L * L * L);
  int T = (int)lround((double)pref * 0.5 / std::max(rho, 1e-9));
  T = std::max(1, std::min(T, pref));
  T = std::min<int>(T, (int)n_cells - 2);
  return std::max(1, std::min(T, kMaxTileT));
}

// Replica index of every global tile (tiles are the replicas' ranges in order), for the kernels.
static int upload_tile_rep(ljmd_batch* b) {
  std::vector<int32_t> tr((size_t)b->caps.ntiles);
  for (int r = 0; r < b->R; ++r) {
    const ReplicaGeo& rg = b->reps_h[r];
    const int64_t nt = (int64_t)rg.n * rg.n * rg.ntz;
    for (int64_t t = 0; t < nt; ++t) tr[(size_t)(rg.tile_base + t)] = r;
  }
  BTRY(balloc(&b->tile_rep, tr.size()));
  BK(cudaMemcpy(b->tile_rep, tr.data(), sizeof(int32_t) * tr.size(), cudaMemcpyHostToDevice));
  return LJ_OK;
}

// Coefficients of the truncation terms of Eq. 2 (Sec. 2.1), as in the single-system path.
static void batch_truncation(double x, int mode, double* c2, double* c0) {
  const double ix2 = 1.0 / (x * x), ix6 = ix2 * ix2 * ix2, ix8 = ix6 * ix2, ix12 = ix6 * ix6, ix14 = ix12 * ix2;
  if (mode == LJ_TRUNC_QUADRATIC) {
    *c2 = 6.0 * ix14 - 3.0 * ix8;
    *c0 = 4.0 * ix6 - 7.0 * ix12;
  } else if (mode == LJ_TRUNC_SHIFT) {
    *c2 = 0.0;
    *c0 = ix6 - ix12;
  } else {
    *c2 = 0.0;
    *c0 = 0.0;
  }
}

// Per-replica boxes, grids and tiles (global ranges in replica order); the constants shared by
// the batch (offset 2^p above the largest box, band of the exact list test, displacement limit).
static int setup_replicas(ljmd_batch* b) {
  const ljmd_params& p = b->prm;
  const double rs = p.cutoff + p.margin;
  b->rs = rs;
  double Lmax = 0.0;
  for (double L : b->box) Lmax = std::max(Lmax, L);
  int pw = 2;
  while (ldexp(1.0, pw) < Lmax + p.margin + 1.0 || ldexp(1.0, pw - 1) < p.margin + 1.0) ++pw;
  b->pw = pw;
  b->offset = ldexp(1.0, pw);
  // one fixed-point unit u = 2^-qk for the batch, with 2^31 u above two cells of the coarsest
  // replica grid plus the drift since the build (the single-system rule, over all replicas)
  double W = 0.0;
  for (double L : b->box) {
    const double nr = std::max(1.0, floor(L / rs));
    W = std::max(W, 2.0 * L / nr + 2.0 * p.margin + 1.0);
  }
  int qk = 31 - (int)ceil(log2(W));
  if (qk > 30) qk = 30;
  b->reps_h.assign(b->R, ReplicaGeo{});
  int64_t tiles = 0, cells = 0;
  for (int r = 0; r < b->R; ++r) {
    const double L = b->box[r];
    if (!(L >= 2.0 * (rs + p.margin)) || !isfinite(L)) return LJ_EINVAL;
    int64_t n = (int64_t)floor(L / rs);
    if (n > 1024) n = 1024;
    // Two cells per side (L / r_s below 3): the neighbour columns and cells of a tile alias, so the
    // tile stages a cell twice with different periodic images.  L >= 2 (r_s + margin) keeps at most
    // one image of a particle within r_s + margin of any key, so each partner is still listed once
    // (by the image the exact distance test accepts) and the force takes that image.
    if (n < 2) return LJ_ERANGE;
    ReplicaGeo& rg = b->reps_h[r];
    Geom& g = rg.g;
    g.L = L;
    g.half_L = 0.5 * L;
    g.offset = b->offset;
    g.inv_h = (double)n / L;
    g.n = (int32_t)n;
    g.p = pw;
    const double q = ldexp(1.0, pw - 23);
    const double Lhi = floor(L / q) * q;
    g.L_hi = (float)Lhi;
    g.L_lo = (float)(L - Lhi);
    g.inv_L = (float)(1.0 / L);
    g.inv_L64 = 1.0 / L;
    g.qk = qk;
    g.qu = (float)ldexp(1.0, -qk);
    g.Lq = (uint32_t)fmod(nearbyint(ldexp(L, qk)), 4294967296.0);
    g.q_inv_L = (float)(ldexp(1.0, -qk) / L);
    const int T = replica_tile(b->tile_T, n, b->count[r], L);
    rg.n = (int32_t)n;
    rg.T = T;
    rg.ntz = (int32_t)((n + T - 1) / T);
    rg.tile_base = tiles;
    rg.cell_base = cells;
    rg.base = b->base[r];
    rg.count = b->count[r];
    tiles += n * n * rg.ntz;
    cells += n * n * n;
  }
  if (cells > 0xffffffffLL || tiles > 0x7fffffffLL) return LJ_ERANGE;
  b->g0 = b->reps_h[0].g;
  b->ncells = cells;
  b->caps.n = 0;
  b->caps.T = 0;
  b->caps.ntz = 0;
  b->caps.whole = 0;
  b->caps.ntiles = tiles;
  double c2, c0;
  batch_truncation(p.cutoff / p.sigma, p.truncation, &c2, &c0);
  LJConst& c = b->c;
  c.eps = p.eps;
  c.sigma = p.sigma;
  c.sig2 = p.sigma * p.sigma;
  c.rc2 = p.cutoff * p.cutoff;
  c.c2 = c2;
  c.c0 = c0;
  c.inv_sigma = 1.0 / c.sigma;
  c.c2s = c.c2 / c.sig2;
  c.inv_sigmaf = (float)c.inv_sigma;
  c.c2sf = (float)c.c2s;
  c.f24 = (float)(24.0 * p.eps);
  c.f48 = (float)(48.0 * p.eps);
  c.f8c2 = (float)(8.0 * p.eps * c2 / c.sig2);
  c.sig2f = (float)c.sig2;
  c.rc2f = (float)c.rc2;
  c.e4 = (float)(4.0 * p.eps);
  c.c2f = (float)(c2 / c.sig2);
  c.c0f = (float)c0;
  c.f24q = ldexpf(c.f24, qk);
  c.f48q = ldexpf(c.f48, qk);
  c.f8c2q = ldexpf(c.f8c2, -qk);
  c.sig2q = ldexpf(c.sig2f, 2 * qk);
  c.rc2q = ldexpf(c.rc2f, 2 * qk);
  c.c2q = ldexpf(c.c2f, -2 * qk);
  // band of the FP32 list filter and the displacement limit: the single-system derivation with
  // the batch's common p and u
  const double eps = ldexp(1.0, pw - 22) + ldexp(1.0, pw - 24);
  const double bound = eps * (2.0 * sqrt(3.0) * rs + 3.0 * eps) + 4.0 * 1.2e-7 * rs * rs;
  const double band = 2.0 * bound + 1e-6 * rs * rs;
  b->band.rs2 = rs * rs;
  b->band.lo = (float)(rs * rs - band);
  b->band.hi = (float)(rs * rs + band);
  b->disp_limit = 0.5 * p.margin - (2.0 * sqrt(3.0) * ldexp(1.0, -qk) + 1e-6 * (0.5 * p.margin) + 1e-9);
  BTRY(balloc(&b->reps, b->R));
  BK(cudaMemcpyAsync(b->reps, b->reps_h.data(), sizeof(ReplicaGeo) * b->R, cudaMemcpyHostToDevice, b->st));
  BTRY(upload_tile_rep(b));
  BTRY(balloc(&b->cell_count, b->ncells));
  BTRY(balloc(&b->cell_start, b->ncells + 1));
  BTRY(balloc(&b->cell_fill, b->ncells));
  BTRY(balloc(&b->scan_tmp, scan_tmp_words(b->ncells)));
  BTRY(balloc(&b->tile_list, (size_t)tiles));
  return LJ_OK;
}

// The rebuild of every replica's cell sort and list: fold, label, counting sort, reorder, shadow,
// list.  With pred non-null each kernel runs only if *pred is set (graph form).
static int enqueue_rebuild(ljmd_batch* b, const int* pred) {
  const int64_t N = b->N;
  cudaStream_t st = b->st;
  // zero fills are predicated too: the counters of the last construction must survive skipped ones
  launch_zero_words(b->cell_count, sizeof(uint32_t) * b->ncells, pred, st);
  launch_wrap_label_batch(b->x, b->img, N, b->rep_of, b->reps, b->offset, b->cell_of, b->cell_count, b->status, pred,
                          st);
  b->launches += 1 + launch_scan_u32(b->cell_count, b->cell_start, b->ncells, b->scan_tmp, st, pred);
  launch_zero_words(b->cell_fill, sizeof(uint32_t) * b->ncells, pred, st);
  launch_scatter(b->cell_of, b->cell_start, b->cell_fill, b->perm, N, st, pred);
  launch_cell_rank(b->cell_start, b->ncells, b->perm, b->id, b->perm_id, st, pred);
  launch_gather_state(b->perm_id, N, b->x, b->x_alt, b->v, b->v_alt, b->id, b->id_alt, b->img, b->img_alt, nullptr,
                      nullptr, 0, st, pred);
  launch_copy_words(b->x_alt, b->x, 24 * N, pred, st);
  launch_copy_words(b->v_alt, b->v, 24 * N, pred, st);
  launch_copy_words(b->id_alt, b->id, 4 * N, pred, st);
  launch_copy_words(b->img_alt, b->img, 12 * N, pred, st);
  launch_shadow_all(b->x, N, 1, b->g0.qk, b->hi, b->xq, nullptr, b->ref, st, pred);
  launch_zero_words(b->counter, 2 * sizeof(unsigned long long), pred, st);
  launch_zero_words(b->sizes, 4 * sizeof(unsigned int), pred, st);
  launch_list_batch(b->hi, b->x, b->cell_start, N, b->g0, b->caps, b->band, b->rows, b->tile_list, b->ent,
                    (uint64_t)b->ent_cap, b->counter, b->sizes + 3, b->status, b->reps, b->R, b->tile_rep, pred, st);
  b->launches += 14;
  BKL();
  return LJ_OK;
}

static int read_status(ljmd_batch* b, int32_t* w) {
  BK(cudaMemcpyAsync(b->h_u64, b->status, sizeof(int32_t), cudaMemcpyDeviceToHost, b->st));
  BK(cudaStreamSynchronize(b->st));
  memcpy(w, b->h_u64, sizeof(int32_t));
  return LJ_OK;
}

// Host-driven construction (no predicate): measures the tiles, sizes the capacities with headroom
// for the steps that follow (inside a graph nothing can grow), builds and checks the list.
static int host_build(ljmd_batch* b) {
  cudaStream_t st = b->st;
  drop_graph(b);
  // sort first with provisional capacities, so that the tile measurement sees the new cells
  BK(cudaMemsetAsync(b->cell_count, 0, sizeof(uint32_t) * b->ncells, st));
  launch_wrap_label_batch(b->x, b->img, b->N, b->rep_of, b->reps, b->offset, b->cell_of, b->cell_count, b->status,
                          nullptr, st);
  b->launches += 1 + launch_scan_u32(b->cell_count, b->cell_start, b->ncells, b->scan_tmp, st);
  BK(cudaMemsetAsync(b->sizes, 0, 4 * sizeof(unsigned int), st));
  launch_tile_sizes_batch(b->cell_start, b->caps, b->reps, b->R, b->tile_rep, b->sizes, st);
  b->launches += 1;
  BKL();
  BK(cudaMemcpyAsync(b->h_u64, b->sizes, 2 * sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
  BK(cudaStreamSynchronize(st));
  unsigned int staged, own;
  memcpy(&staged, (char*)b->h_u64, 4);
  memcpy(&own, (char*)b->h_u64 + 4, 4);
  // headroom for the density fluctuations of the steps between host constructions
  b->caps.max_staged = (int32_t)std::min<double>(65535.0, ceil(staged * 1.3) + 32);
  b->caps.max_own = (int32_t)(ceil(own * 1.4) + 16);
  b->caps.max_chunks = 1;
  if (staged > 65535) return LJ_ERANGE;
  int dev = 0, smem_max = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (batch_list_smem_bytes(b->caps) > (size_t)smem_max) return LJ_ERANGE;
  if (b->ent_cap == 0) {
    double est = 0.0;
    for (int r = 0; r < b->R; ++r) {
      const double L = b->box[r];
      est += (double)b->count[r] * 4.18879 * b->rs * b->rs * b->rs * (double)b->count[r] / (L * L * L);
    }
    b->ent_cap = (size_t)(est * 1.5) + 8 * (size_t)b->caps.ntiles + 65536;
    BTRY(balloc(&b->ent, b->ent_cap));
  }
  b->caps.max_list = 0;
  for (int attempt = 0; attempt < 2; ++attempt) {
    BK(cudaMemsetAsync(b->status, 0, sizeof(int32_t), st));
    BTRY(enqueue_rebuild(b, nullptr));
    BK(cudaMemcpyAsync(b->h_u64, b->counter, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    BK(cudaMemcpyAsync(b->h_u64 + 2, b->sizes + 3, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    BK(cudaStreamSynchronize(st));
    const unsigned long long total = b->h_u64[0], actual = b->h_u64[1];
    unsigned int maxlist;
    memcpy(&maxlist, b->h_u64 + 2, 4);
    if (total > 4294967295ULL) return LJ_ERANGE;
    if (total <= b->ent_cap) {
      int32_t w = 0;
      BTRY(read_status(b, &w));
      if (w) {
        fprintf(stderr, "ljmd_batch: list construction raised status %d\n", w);
        return LJ_EDEVICE;
      }
      b->list_entries = total;
      b->list_actual = actual;
      // capacities for the following device-side rebuilds
      b->caps.max_list = (int32_t)(((unsigned)ceil(maxlist * 1.4) + 64u + 7u) & ~7u);
      if (b->ent_cap < (size_t)(total * 1.3) + 65536) {
        b->ent_cap = (size_t)(total * 1.4) + 65536;
        BTRY(balloc(&b->ent, b->ent_cap));
        continue;  // construct again into the larger array
      }
      break;
    }
    b->ent_cap = (size_t)(total * 1.4) + 65536;
    BTRY(balloc(&b->ent, b->ent_cap));
    if (attempt == 1) return LJ_EDEVICE;
  }
  if (b->caps.max_list == 0) return LJ_EDEVICE;
  {  // list segments beyond what fits next to the staged positions are read from HBM
    TileArgs tz = b->caps;
    tz.list_cap = 0;
    const size_t base_bytes = batch_force_smem_bytes(tz);
    if (base_bytes > (size_t)smem_max) return LJ_ERANGE;
    // room for the list next to the positions so that 4 CTAs share an SM where possible
    const int64_t target = std::max<int64_t>((int64_t)base_bytes + 4096, 54 * 1024);
    const int64_t room = (std::min<int64_t>(smem_max, target) - (int64_t)base_bytes) / 2 - 16;
    b->caps.list_cap = (int32_t)std::max<int64_t>(0, std::min<int64_t>(b->caps.max_list, room) & ~(int64_t)7);
  }
  b->have_list = true;
  b->forces_current = false;
  b->host_rebuilds += 1;
  return LJ_OK;
}

static int enqueue_force(ljmd_batch* b, bool energy) {
  if (energy) BK(cudaMemsetAsync(b->e_rep, 0, 2 * sizeof(double) * b->R, b->st));
  launch_force_batch(b->lanes, energy ? 1 : 0, b->xq, b->cell_start, b->N, b->caps, b->c, b->rows,
                     b->tile_list, b->ent, b->f, b->e_rep, b->status, b->reps, b->R, b->tile_rep, b->st);
  b->launches += 1;
  BKL();
  return LJ_OK;
}

// k steps of velocity-Verlet (v at the full step on entry and on exit), no host synchronisation:
// kick-drift with the displacement maximum, device flag, predicated rebuild, force; final kick.
static int enqueue_steps(ljmd_batch* b, double dt, int64_t k) {
  const double h = 0.5 * dt;
  const float limit2 = (float)(b->disp_limit * b->disp_limit);
  for (int64_t s = 0; s < k; ++s) {
    BK(cudaMemsetAsync(b->dmax, 0, 2 * sizeof(uint32_t), b->st));
    IntegrateArgs a{s == 0 ? 0.0 : h, h, dt, 0, 1, 0, b->g0.qk};
    launch_integrate(LJ_MIXED, b->x, b->v, b->f, b->xq, b->ref, b->N, a, nullptr, b->dmax, b->status, StepFinish{}, b->st);
    launch_rebuild_flag(b->dmax, limit2, b->flag, b->d_rebuilds, b->st);
    b->launches += 2;
    BTRY(enqueue_rebuild(b, b->flag));
    BTRY(enqueue_force(b, false));
  }
  IntegrateArgs a{h, 0.0, 0.0, 0, 0, 0, b->g0.qk};
  launch_integrate(LJ_MIXED, b->x, b->v, b->f, b->xq, b->ref, b->N, a, nullptr, b->dmax, b->status, StepFinish{}, b->st);
  b->launches += 1;
  BKL();
  return LJ_OK;
}

static int check_batch_status(ljmd_batch* b) {
  int32_t w = 0;
  BTRY(read_status(b, &w));
  if (w) {
    fprintf(stderr, "ljmd_batch: device status %d (1 non-finite, 2 list overflow, 4 timeout, 8 tile capacity)\n", w);
    return LJ_EDEVICE;
  }
  return LJ_OK;
}

extern "C" {

int ljmd_batch_create(ljmd_batch** out, const ljmd_params* p, int32_t replicas, const int64_t* n, const double* box,
                      void* cuda_stream) {
  if (!out || !p || replicas <= 0 || !n || !box) return LJ_EINVAL;
  *out = nullptr;
  if (!(p->cutoff > 0.0) || !(p->margin >= 0.0) || !(p->eps > 0.0) || !(p->sigma > 0.0)) return LJ_EINVAL;
  if (p->truncation < 0 || p->truncation > 2) return LJ_EINVAL;
  ljmd_batch* b = new ljmd_batch();
  b->prm = *p;
  b->user_st = (cudaStream_t)cuda_stream;
  if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->user_ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    free_batch(b);
    delete b;
    return LJ_EDEVICE;
  }
  b->R = replicas;
  if (p->lanes == 2 || p->lanes == 4 || p->lanes == 8) b->lanes = p->lanes;
  int64_t N = 0;
  for (int r = 0; r < replicas; ++r) {
    if (n[r] <= 0) {
      delete b;
      return LJ_EINVAL;
    }
    b->base.push_back(N);
    b->count.push_back(n[r]);
    b->box.push_back(box[r]);
    N += n[r];
  }
  if (N > 1000000000LL) {
    delete b;
    return LJ_ERANGE;
  }
  b->N = N;
  cudaGetDevice(&b->device);
  int r = setup_replicas(b);
  auto A = [&](auto** ptr, size_t cnt) {
    if (r == LJ_OK) r = balloc(ptr, cnt);
  };
  A(&b->x, 3 * N);
  A(&b->v, 3 * N);
  A(&b->x_alt, 3 * N);
  A(&b->v_alt, 3 * N);
  A(&b->f, N);
  A(&b->hi, N);
  A(&b->xq, N);
  A(&b->ref, N);
  A(&b->id, N);
  A(&b->id_alt, N);
  A(&b->img, 3 * N);
  A(&b->img_alt, 3 * N);
  A(&b->rep_of, N);
  A(&b->cell_of, N);
  A(&b->perm, N);
  A(&b->perm_id, N);
  A(&b->rows, N);
  A(&b->e_rep, 2 * (size_t)replicas);
  A(&b->ke_rep, (size_t)replicas);
  A(&b->status, 1);
  A(&b->dmax, 2);
  A(&b->flag, 1);
  A(&b->d_rebuilds, 1);
  A(&b->counter, 2);
  A(&b->sizes, 4);
  if (r == LJ_OK && cudaMallocHost(&b->h_f64, 64) != cudaSuccess) r = LJ_ENOMEM;
  if (r == LJ_OK && cudaMallocHost(&b->h_u64, 64) != cudaSuccess) r = LJ_ENOMEM;
  if (r == LJ_OK) {
    std::vector<int32_t> rep(N);
    for (int q = 0; q < replicas; ++q)
      for (int64_t i = 0; i < n[q]; ++i) rep[b->base[q] + i] = q;
    if (cudaMemcpyAsync(b->rep_of, rep.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, b->st) != cudaSuccess ||
        cudaMemsetAsync(b->status, 0, 4, b->st) != cudaSuccess ||
        cudaMemsetAsync(b->d_rebuilds, 0, 8, b->st) != cudaSuccess ||
        cudaStreamSynchronize(b->st) != cudaSuccess)
      r = LJ_EDEVICE;
  }
  if (r != LJ_OK) {
    free_batch(b);
    delete b;
    cudaGetLastError();
    return r;
  }
  *out = b;
  return LJ_OK;
}

void ljmd_batch_destroy(ljmd_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->st);
  free_batch(b);
  cudaGetLastError();
  delete b;
}

int ljmd_batch_set_state(ljmd_batch* b, const double* x, const double* v, int32_t on_device) {
  if (!b || !x) return LJ_EINVAL;
  if (b->broken) return LJ_EDEVICE;
  BTRY(join_user(b));
  const int64_t N = b->N;
  cudaStream_t st = b->st;
  const double* xs = x;
  const double* vs = v;
  if (!on_device) {
    BK(cudaMemcpyAsync(b->x_alt, x, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, st));
    xs = b->x_alt;
    if (v) {
      BK(cudaMemcpyAsync(b->v_alt, v, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, st));
      vs = b->v_alt;
    }
  }
  launch_load_batch(xs, vs, b->x, b->v, b->id, b->img, N, b->rep_of, b->reps, b->offset, st);
  b->launches += 1;
  BKL();
  BK(cudaMemsetAsync(b->f, 0, sizeof(float4) * N, st));
  BK(cudaMemsetAsync(b->status, 0, 4, st));
  if (!on_device) BK(cudaStreamSynchronize(st));
  b->have_state = true;
  b->have_list = false;
  b->forces_current = false;
  b->steps = 0;
  return LJ_OK;
}

int ljmd_batch_step(ljmd_batch* b, double dt, int64_t nsteps, int32_t graph_steps) {
  if (!b || nsteps < 0 || graph_steps < 0 || !isfinite(dt)) return LJ_EINVAL;
  if (b->broken) return LJ_EDEVICE;
  BTRY(join_user(b));
  if (!b->have_state) return LJ_ESTATE;
  if (nsteps == 0) return LJ_OK;
  if (!b->have_list) BTRY(host_build(b));
  if (!b->forces_current) {
    BTRY(enqueue_force(b, false));
    b->forces_current = true;
  }
  int64_t done = 0;
  if (graph_steps > 0 && nsteps >= graph_steps) {
    if (!b->gexec || b->g_steps != graph_steps || b->g_dt != dt) {
      drop_graph(b);
      // one plain step first sets every kernel attribute outside the capture
      BTRY(enqueue_steps(b, dt, 1));
      done += 1;
      cudaGraph_t graph = nullptr;
      BK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
      const int64_t launches0 = b->launches;
      int rc = enqueue_steps(b, dt, graph_steps);
      cudaError_t ec = cudaStreamEndCapture(b->st, &graph);
      if (rc != LJ_OK) return rc;
      BK(ec);
      b->g_launches = b->launches - launches0;
      b->launches = launches0;  // counted per replay below
      cudaGraphExec_t exec = nullptr;
      cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      BK(ei);
      b->gexec = exec;
      b->g_steps = graph_steps;
      b->g_dt = dt;
    }
    while (nsteps - done >= graph_steps) {
      BK(cudaGraphLaunch(b->gexec, b->st));
      b->launches += b->g_launches;
      done += graph_steps;
    }
  }
  if (nsteps > done) BTRY(enqueue_steps(b, dt, nsteps - done));
  b->steps += nsteps;
  return check_batch_status(b);
}

int ljmd_batch_energies(ljmd_batch* b, double* pe, double* ke, double* virial) {
  if (!b) return LJ_EINVAL;
  if (b->broken) return LJ_EDEVICE;
  BTRY(join_user(b));
  if (!b->have_state) return LJ_ESTATE;
  if (!b->have_list) BTRY(host_build(b));
  BTRY(enqueue_force(b, true));
  b->forces_current = true;
  BK(cudaMemsetAsync(b->ke_rep, 0, sizeof(double) * b->R, b->st));
  launch_replica_ke(b->v, b->N, b->reps, b->R, b->ke_rep, b->st);
  b->launches += 1;
  BKL();
  std::vector<double> e(2 * (size_t)b->R), k((size_t)b->R);
  BK(cudaMemcpyAsync(e.data(), b->e_rep, sizeof(double) * 2 * b->R, cudaMemcpyDeviceToHost, b->st));
  BK(cudaMemcpyAsync(k.data(), b->ke_rep, sizeof(double) * b->R, cudaMemcpyDeviceToHost, b->st));
  BK(cudaStreamSynchronize(b->st));
  for (int r = 0; r < b->R; ++r) {
    if (pe) pe[r] = e[2 * r];
    if (virial) virial[r] = e[2 * r + 1];
    if (ke) ke[r] = k[r];
  }
  return check_batch_status(b);
}

int ljmd_batch_get_state(ljmd_batch* b, double* x, double* v, double* f, int32_t on_device) {
  if (!b) return LJ_EINVAL;
  if (b->broken) return LJ_EDEVICE;
  BTRY(join_user(b));
  if (!b->have_state) return LJ_ESTATE;
  const int64_t N = b->N;
  cudaStream_t st = b->st;
  double* tmp = b->x_alt;  // free between rebuilds
  if (x) {
    double* dst = on_device ? x : tmp;
    launch_scatter_back_f64x3(b->x, dst, b->id, N, b->offset, st);
    if (!on_device) BK(cudaMemcpyAsync(x, dst, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, st));
  }
  if (v) {
    double* dst = on_device ? v : tmp;
    launch_scatter_back_f64x3(b->v, dst, b->id, N, 0.0, st);
    if (!on_device) BK(cudaMemcpyAsync(v, dst, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, st));
  }
  if (f) {
    if (!b->forces_current) {
      if (!b->have_list) BTRY(host_build(b));
      BTRY(enqueue_force(b, false));
      b->forces_current = true;
    }
    double* dst = on_device ? f : tmp;
    launch_scatter_back_f32x4_to_f64x3(b->f, dst, b->id, N, st);
    if (!on_device) BK(cudaMemcpyAsync(f, dst, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, st));
  }
  BKL();
  BK(cudaStreamSynchronize(st));
  return check_batch_status(b);
}

int ljmd_batch_get_pairs(ljmd_batch* b, int32_t replica, int64_t* ij, int64_t cap, int64_t* npairs) {
  if (!b || !npairs || replica < 0 || replica >= b->R || cap < 0 || (cap > 0 && !ij)) return LJ_EINVAL;
  if (b->broken) return LJ_EDEVICE;
  if (!b->have_state) return LJ_ESTATE;
  if (!b->have_list) BTRY(host_build(b));
  cudaStream_t st = b->st;
  // list size as built last (device-side rebuilds update the counter)
  BK(cudaMemcpyAsync(b->h_u64, b->counter, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  BK(cudaStreamSynchronize(st));
  const uint64_t E = b->h_u64[0];
  const ReplicaGeo& rg = b->reps_h[replica];
  TileArgs ta = b->caps;
  ta.n = rg.n;
  ta.T = rg.T;
  ta.ntz = rg.ntz;
  ta.whole = 0;
  ta.ntiles = (int64_t)rg.n * rg.n * rg.ntz;
  uint32_t* d_pairs = nullptr;
  BTRY(balloc(&d_pairs, 2 * E + 2));
  std::vector<uint32_t> pr(2 * E + 2);
  std::vector<uint2> rows((size_t)rg.count);
  std::vector<int32_t> id((size_t)rg.count);
  cudaError_t e1 = cudaMemsetAsync(d_pairs, 0xff, sizeof(uint32_t) * (2 * E + 2), st);
  if (e1 == cudaSuccess) {
    launch_list_decode(b->cell_start + rg.cell_base, b->N, ta, b->rows, b->ent, E, d_pairs, b->status, st);
    b->launches += 1;
    e1 = cudaGetLastError();
  }
  if (e1 == cudaSuccess && E)
    e1 = cudaMemcpyAsync(pr.data(), d_pairs, sizeof(uint32_t) * 2 * E, cudaMemcpyDeviceToHost, st);
  if (e1 == cudaSuccess)
    e1 = cudaMemcpyAsync(rows.data(), b->rows + rg.base, sizeof(uint2) * rg.count, cudaMemcpyDeviceToHost, st);
  if (e1 == cudaSuccess)
    e1 = cudaMemcpyAsync(id.data(), b->id + rg.base, sizeof(int32_t) * rg.count, cudaMemcpyDeviceToHost, st);
  if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(st);
  cudaFree(d_pairs);
  if (e1 != cudaSuccess) {
    b->broken = true;
    return LJ_EDEVICE;
  }
  std::vector<std::pair<int64_t, int64_t>> pairs;
  for (int64_t s = 0; s < rg.count; ++s) {
    const uint2 row = rows[s];
    if ((uint64_t)row.x + row.y > E) return LJ_EDEVICE;
    for (unsigned e = 0; e < row.y; ++e) {
      const uint32_t gi = pr[2 * ((size_t)row.x + e)], gj = pr[2 * ((size_t)row.x + e) + 1];
      if (gi != (uint32_t)(rg.base + s) || gj < (uint64_t)rg.base || gj >= (uint64_t)(rg.base + rg.count))
        return LJ_EDEVICE;
      const int64_t a = id[s] - rg.base, c = id[gj - rg.base] - rg.base;
      if (a < c) pairs.emplace_back(a, c);
    }
  }
  std::sort(pairs.begin(), pairs.end());
  *npairs = (int64_t)pairs.size();
  const int64_t m = std::min<int64_t>(cap, (int64_t)pairs.size());
  for (int64_t k = 0; k < m; ++k) {
    ij[2 * k] = pairs[k].first;
    ij[2 * k + 1] = pairs[k].second;
  }
  return check_batch_status(b);
}

int ljmd_batch_get_stats(ljmd_batch* b, ljmd_batch_stats* out) {
  if (!b || !out) return LJ_EINVAL;
  memset(out, 0, sizeof(*out));
  out->replicas = b->R;
  out->n = b->N;
  out->steps = b->steps;
  out->tiles = b->caps.ntiles;
  out->cells = b->ncells;
  out->tile_cells = b->tile_T;
  out->lanes = b->lanes;
  out->kernel_launches = b->launches;
  if (b->broken) return LJ_EDEVICE;
  cudaStream_t st = b->st;
  if (cudaMemcpyAsync(b->h_u64, b->counter, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(b->h_u64 + 2, b->d_rebuilds, sizeof(long long), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(b->h_u64 + 3, b->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    b->broken = true;
    return LJ_EDEVICE;
  }
  out->list_entries = (int64_t)b->h_u64[1];
  out->rebuilds = b->host_rebuilds + (int64_t)b->h_u64[2];
  int32_t w;
  memcpy(&w, b->h_u64 + 3, 4);
  out->status_word = w;
  return LJ_OK;
}

int ljmd_batch_set_tuning(ljmd_batch* b, int32_t tile_cells, int32_t lanes) {
  if (!b) return LJ_EINVAL;
  if (b->broken) return LJ_EDEVICE;
  if (tile_cells < 0 || tile_cells > kMaxTileT) return LJ_EINVAL;
  if (!(lanes == 0 || lanes == 2 || lanes == 4 || lanes == 8)) return LJ_EINVAL;
  if (lanes) b->lanes = lanes;
  if (tile_cells && tile_cells != b->tile_T) {
    b->tile_T = tile_cells;
    for (ReplicaGeo& rg : b->reps_h) {
      rg.T = replica_tile(tile_cells, rg.n, rg.count, rg.g.L);
      rg.ntz = (rg.n + rg.T - 1) / rg.T;
    }
    int64_t tiles = 0;
    for (ReplicaGeo& rg : b->reps_h) {
      rg.tile_base = tiles;
      tiles += (int64_t)rg.n * rg.n * rg.ntz;
    }
    b->caps.ntiles = tiles;
    BK(cudaMemcpyAsync(b->reps, b->reps_h.data(), sizeof(ReplicaGeo) * b->R, cudaMemcpyHostToDevice, b->st));
    BTRY(balloc(&b->tile_list, (size_t)tiles));
    BTRY(upload_tile_rep(b));
    b->have_list = false;
    b->forces_current = false;
  }
  drop_graph(b);
  return LJ_OK;
}

// Mean device time of one force launch over all replicas at the current positions and lists:
// one warm-up launch, then `trials` launches between CUDA events on the batch's stream.  Forces are
// recomputed (the state is otherwise unchanged).
int ljmd_batch_time_force(ljmd_batch* b, int32_t trials, double* ms_per_launch) {
  if (!b || trials <= 0 || !ms_per_launch) return LJ_EINVAL;
  if (b->broken) return LJ_EDEVICE;
  BTRY(join_user(b));
  if (!b->have_state) return LJ_ESTATE;
  if (!b->have_list) BTRY(host_build(b));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return LJ_EDEVICE;
  }
  int rc = enqueue_force(b, false);
  if (rc == LJ_OK && cudaEventRecord(e0, b->st) != cudaSuccess) rc = LJ_EDEVICE;
  for (int k = 0; k < trials && rc == LJ_OK; ++k) rc = enqueue_force(b, false);
  float ms = 0.f;
  if (rc == LJ_OK && (cudaEventRecord(e1, b->st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                      cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
    rc = LJ_EDEVICE;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != LJ_OK) {
    b->broken = rc == LJ_EDEVICE;
    return rc;
  }
  b->forces_current = true;
  *ms_per_launch = (double)ms / trials;
  return check_batch_status(b);
}

// Project autotuner: for each (tile_cells, lanes) candidate, construct the list at the current
// positions and time `trials` force launches plus the construction (CUDA events on the batch's
// stream); the cost is force + construction / 10 (a typical list lifetime).  The fastest is kept.
// Positions and velocities are unchanged (constructions only reorder).
int ljmd_batch_autotune(ljmd_batch* b, int32_t trials, int32_t* best_tile, int32_t* best_lanes, double* best_ms) {
  if (!b || trials <= 0) return LJ_EINVAL;
  if (b->broken) return LJ_EDEVICE;
  if (!b->have_state) return LJ_ESTATE;
  const int tiles[] = {2, 3, 4, 6};
  const int lanes_c[] = {2, 4, 8};
  cudaEvent_t e0, e1, e2;
  BK(cudaEventCreate(&e0));
  BK(cudaEventCreate(&e1));
  BK(cudaEventCreate(&e2));
  double best = 1e300;
  int bt = b->tile_T, bl = b->lanes;
  int rc = LJ_OK;
  for (int T : tiles) {
    if ((rc = ljmd_batch_set_tuning(b, T, 0)) != LJ_OK) break;
    if (cudaEventRecord(e0, b->st) != cudaSuccess) {
      rc = LJ_EDEVICE;
      break;
    }
    if ((rc = host_build(b)) != LJ_OK) break;
    cudaEventRecord(e1, b->st);
    cudaEventSynchronize(e1);
    float build_ms = 0.f;
    cudaEventElapsedTime(&build_ms, e0, e1);
    for (int L : lanes_c) {
      b->lanes = L;
      if ((rc = enqueue_force(b, false)) != LJ_OK) break;  // warm-up (kernel attributes)
      cudaEventRecord(e1, b->st);
      for (int k = 0; k < trials && rc == LJ_OK; ++k) rc = enqueue_force(b, false);
      cudaEventRecord(e2, b->st);
      if (cudaEventSynchronize(e2) != cudaSuccess) rc = LJ_EDEVICE;
      if (rc != LJ_OK) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e1, e2);
      const double cost = ms / trials + build_ms / 10.0;
      if (cost < best) {
        best = cost;
        bt = T;
        bl = L;
      }
    }
    if (rc != LJ_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  if (rc != LJ_OK) return rc;
  BTRY(ljmd_batch_set_tuning(b, bt, bl));
  BTRY(host_build(b));
  b->forces_current = false;
  if (best_tile) *best_tile = bt;
  if (best_lanes) *best_lanes = bl;
  if (best_ms) *best_ms = best;
  return check_batch_status(b);
}

}  // extern "C"
