// C ABI of libljmd (declared in include/ljmd.h): handle management and the host-side
// orchestration of the hot path.  Every step of the computation runs in the kernels of the
// other translation units; this file only sizes buffers, launches and reads back scalars.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ljmd_internal.h"

using namespace ljmd;

struct ljmd_sys {
  int device = 0;
  cudaStream_t st = nullptr;
  ljmd_params prm{};
  int precision = LJ_MIXED;
  bool broken = false;

  // particles and geometry
  int64_t n = 0;
  double L = 0.0;
  Geom g{};
  LJConst c{};
  ListBand band{};
  double rs = 0.0;
  int64_t ncells = 0;
  double disp_limit = 0.0;  // rebuild when the measured displacement exceeds this

  // bookkeeping
  bool have_list = false;
  bool forces_current = false;
  int64_t pe_step = -1;      // state index whose PE/virial partials are in part_force
  int64_t energy_step = -1;  // state index of the energies in d_energies
  int64_t steps = 0, rebuilds = 0;
  uint64_t list_entries = 0;     // reserved entries (tile segments padded to 8)
  uint64_t list_actual = 0;      // entries actually listed
  double last_dmax = 0.0;
  int nb_force = 0;
  double* log_ptr = nullptr;
  int64_t log_cap = 0;

  // device buffers (sorted order)
  double *x = nullptr, *v = nullptr, *x_alt = nullptr, *v_alt = nullptr;
  void *f = nullptr, *f_alt = nullptr;
  float4* hi = nullptr;   // FP32 hi parts of the positions (the list construction's filter)
  uint4* xq = nullptr;    // mixed form: fixed-point records of the positions (force and adjoint)
  dvec4* pos64 = nullptr; // FP64 form: position copies for the force and adjoint kernels
  void* ref = nullptr;
  int32_t *id = nullptr, *id_alt = nullptr, *img = nullptr, *img_alt = nullptr;
  uint32_t *cell_of = nullptr, *perm = nullptr, *perm_id = nullptr;  // perm_id: perm ordered by id in each cell
  uint32_t *cell_count = nullptr, *cell_start = nullptr, *cell_fill = nullptr;
  uint2* rows = nullptr;        // per particle: (start, length) of its row in ent
  uint2* tile_list = nullptr;   // per tile: (start, length) of its segment of ent
  int64_t tile_list_cap = 0;
  uint16_t* ent = nullptr;       // SortedList: partner indices into the key's staged tile
  size_t ent_cap = 0;
  TileArgs ta{};
  int tile_T = 0;                // preferred cells per tile along z (0 = default)
  int force_per_sm = 0;          // force CTAs per SM (0 = as many as fit)
  int force_nbuf = 0;            // tile buffers per force CTA (1 or 2; 0 = default)
  bool list_half = false;        // the list form in use (LJ_LIST_AUTO resolved)
  uint32_t* scan_tmp = nullptr;
  size_t scan_tmp_cap = 0;
  int64_t cap_n = 0;       // particle capacity of the per-particle buffers
  int64_t cap_cells = 0;   // capacity of the per-cell buffers
  double *part_force = nullptr, *part_ke = nullptr, *part_misc = nullptr, *d_scalars = nullptr;
  double* d_energies = nullptr;
  int64_t* d_log_count = nullptr;
  int32_t* d_status = nullptr;
  uint32_t* d_dmax = nullptr;
  StepCtl* d_ctl = nullptr;     // device-decided runs: stop flag, stopping step, last maxima, DUTC buffer
  unsigned int* d_ticket = nullptr;  // CTAs of an integrator launch that finished (the last one finishes the step)
  // Capture hook of the trajectory gradient: if set, the unwrapped positions (id order) of every
  // state t reached by a step go to cap_x + 3 n (t - cap_step0).
  double* cap_x = nullptr;
  int64_t cap_step0 = 0;
  StepCtl* h_ctl = nullptr;     // pinned mirror
  int64_t last_build_step = 0;  // sys->steps at the last list construction
  int64_t lifetime_est = 16;    // steps the last list lived (sizes the next device-decided run)
  unsigned long long* d_total64 = nullptr;
  unsigned int* d_sizes = nullptr;
  // profiling: event pairs per phase, resolved when the profile is read
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;  // (phase, (start, stop))
  double prof_ms[5] = {0, 0, 0, 0, 0};
  int64_t prof_n[5] = {0, 0, 0, 0, 0};
  int64_t launches = 0;
  // list validity rule (Sec. 2.3 / Alg. 2)
  int valid_mode = LJ_VALID_HALF_MARGIN;
  int max_ld = 4096;          // N_l of the LDC method
  double dutc_buffer = 0.0;   // buffer_length of the DUTC method
  double last_vmax = 0.0;     // largest drift speed of the last step
  double* xref64 = nullptr;   // FP64 positions the list was built from (LDC)
  int64_t xref_cap = 0;
  int32_t* ldc_list = nullptr;
  unsigned int* d_ldc = nullptr;  // [0] |L_D|, [1] invalid flag
  int64_t ldc_checks = 0, ldc_kept = 0;
  // adjoint pass (allocated on first use)
  dvec4 *adj_w = nullptr, *adj_hw = nullptr, *adj_f = nullptr;
  float4* adj_wf = nullptr;           // FP32 copy of adj_w
  unsigned int* adj_ticket = nullptr;  // CTAs of an adjoint launch that finished
  double* part_adj = nullptr;
  double* d_adj = nullptr;
  int64_t adj_cap = 0;
  // pinned host mirrors
  uint32_t* h_u32 = nullptr;
  double* h_f64 = nullptr;
  int32_t* h_i32 = nullptr;
};

// ----------------------------------------------------------------------------------------------
#define CK(call)                         \
  do {                                   \
    cudaError_t e_ = (call);             \
    if (e_ != cudaSuccess) {             \
      sys->broken = true;                \
      return LJ_EDEVICE;                 \
    }                                    \
  } while (0)
#define CKL() CK(cudaGetLastError())
#define TRY(expr)            \
  do {                       \
    int r_ = (expr);         \
    if (r_ != LJ_OK) return r_; \
  } while (0)

static int dalloc(ljmd_sys* sys, void** p, size_t bytes) {
  if (*p) cudaFree(*p);
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return LJ_ENOMEM;
  }
  (void)sys;
  return LJ_OK;
}
template <class T>
static int dalloc_t(ljmd_sys* sys, T** p, size_t count) {
  return dalloc(sys, (void**)p, count * sizeof(T));
}

static void free_all(ljmd_sys* s) {
  void* ptrs[] = {s->x, s->v, s->x_alt, s->v_alt, s->f, s->f_alt, s->hi, s->xq, s->pos64, s->ref, s->id,
                  s->id_alt, s->img, s->img_alt, s->cell_of, s->perm, s->perm_id, s->cell_count, s->cell_start,
                  s->cell_fill, s->rows, s->tile_list, s->ent, s->scan_tmp, s->part_force, s->part_ke,
                  s->part_misc, s->d_scalars, s->d_energies, s->d_log_count, s->d_status, s->d_dmax, s->d_ctl, s->d_ticket, s->d_total64, s->d_sizes,
                  s->adj_w, s->adj_hw, s->adj_f, s->adj_wf, s->adj_ticket, s->part_adj, s->d_adj, s->xref64, s->ldc_list, s->d_ldc};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (auto& p : s->ev_pending) {
    cudaEventDestroy(p.second.first);
    cudaEventDestroy(p.second.second);
  }
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  if (s->h_u32) cudaFreeHost(s->h_u32);
  if (s->h_f64) cudaFreeHost(s->h_f64);
  if (s->h_i32) cudaFreeHost(s->h_i32);
  if (s->h_ctl) cudaFreeHost(s->h_ctl);
}

enum { PH_FORCE = 0, PH_INTEGRATE = 1, PH_REBUILD = 2, PH_ENERGY = 3, PH_ADJOINT = 4 };

static cudaEvent_t ev_get(ljmd_sys* s) {
  if (!s->ev_pool.empty()) {
    cudaEvent_t e = s->ev_pool.back();
    s->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Scoped phase timer: records a start event now and a stop event at scope exit (profiling only).
struct PhaseTimer {
  ljmd_sys* s;
  int phase;
  cudaEvent_t a = nullptr;
  PhaseTimer(ljmd_sys* s_, int ph) : s(s_), phase(ph) {
    if (s->profiling && (a = ev_get(s))) cudaEventRecord(a, s->st);
  }
  ~PhaseTimer() {
    if (!a) return;
    cudaEvent_t b = ev_get(s);
    if (!b) return;
    cudaEventRecord(b, s->st);
    s->ev_pending.push_back({phase, {a, b}});
  }
};

static void resolve_events(ljmd_sys* s) {
  for (auto& p : s->ev_pending) {
    float ms = 0.0f;
    if (cudaEventSynchronize(p.second.second) == cudaSuccess &&
        cudaEventElapsedTime(&ms, p.second.first, p.second.second) == cudaSuccess) {
      s->prof_ms[p.first] += ms;
      s->prof_n[p.first] += 1;
    }
    cudaGetLastError();
    s->ev_pool.push_back(p.second.first);
    s->ev_pool.push_back(p.second.second);
  }
  s->ev_pending.clear();
}

// Coefficients of the additive truncation terms of Eq. 2 (Sec. 2.1), from V(r_c) = V'(r_c) = 0
// with x = r_c / sigma: c2 = 6 x^-14 - 3 x^-8, c0 = 4 x^-6 - 7 x^-12.  Shift-only: c2 = 0,
// c0 = x^-6 - x^-12.  Plain cut: both zero.
static void truncation_terms(double x, int mode, double* c2, double* c0) {
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

static int check_params(const ljmd_params* p) {
  if (!(p->cutoff > 0.0) || !(p->margin >= 0.0) || !(p->eps > 0.0) || !(p->sigma > 0.0)) return LJ_EINVAL;
  if (p->truncation < 0 || p->truncation > 2) return LJ_EINVAL;
  if (p->list_form != LJ_LIST_FULL && p->list_form != LJ_LIST_HALF && p->list_form != LJ_LIST_AUTO) return LJ_EINVAL;
  if (p->energy_every < 0) return LJ_EINVAL;
  const int l = p->lanes;
  if (!(l == 0 || l == 1 || l == 2 || l == 4 || l == 8 || l == 16 || l == 32)) return LJ_EINVAL;
  return LJ_OK;
}

// How far the measured largest displacement can fall short of the FP64 one.
static double disp_slack(const ljmd_sys* s) {
  if (s->precision != LJ_MIXED) return 1e-12;
  return 2.0 * sqrt(3.0) * (double)s->g.qu + 1e-6 * (0.5 * s->prm.margin) + 1e-9;
}

// Box, cutoff and margin -> grid, offsets, constants.  Requires L >= 2 (r_s + margin) so that a
// listed pair, which can close in by at most the margin, keeps a unique minimum image.
static int setup_geometry(ljmd_sys* s, double L) {
  const ljmd_params& p = s->prm;
  const double rs = p.cutoff + p.margin;
  if (!(L >= 2.0 * (rs + p.margin)) || !isfinite(L)) return LJ_EINVAL;
  s->L = L;
  s->rs = rs;
  int64_t n = (int64_t)floor(L / rs);
  if (n < 1) n = 1;
  if (n > 1024) n = 1024;
  s->ncells = n * n * n;
  int pw = 2;
  while (ldexp(1.0, pw) < L + p.margin + 1.0 || ldexp(1.0, pw - 1) < p.margin + 1.0) ++pw;
  Geom& g = s->g;
  g.L = L;
  g.half_L = 0.5 * L;
  g.offset = ldexp(1.0, pw);
  g.inv_h = (double)n / L;
  g.n = (int32_t)n;
  g.p = pw;
  const double q = ldexp(1.0, pw - 23);
  const double Lhi = floor(L / q) * q;
  g.L_hi = (float)Lhi;
  g.L_lo = (float)(L - Lhi);
  g.inv_L = (float)(1.0 / L);
  g.inv_L64 = 1.0 / L;
  // Fixed-point records (mixed form): u = 2^-qk with 2^31 u above every difference the kernels
  // take: two staged neighbour cells (2 h) or the whole box (fewer than 3 cells per side), plus
  // the drift of both particles since the build and a unit of headroom.
  {
    const double W = (n < 3 ? L : 2.0 * L / (double)n) + 2.0 * p.margin + 1.0;
    int qk = 31 - (int)ceil(log2(W));
    if (qk > 30) qk = 30;
    g.qk = qk;
    const double u = ldexp(1.0, -qk);
    g.qu = (float)u;
    g.Lq = (uint32_t)fmod(nearbyint(ldexp(L, qk)), 4294967296.0);
    g.q_inv_L = (float)(u / L);
  }

  double c2, c0;
  truncation_terms(p.cutoff / p.sigma, p.truncation, &c2, &c0);
  LJConst& c = s->c;
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
  c.f24q = ldexpf(c.f24, g.qk);
  c.f48q = ldexpf(c.f48, g.qk);
  c.f8c2q = ldexpf(c.f8c2, -g.qk);
  c.sig2q = ldexpf(c.sig2f, 2 * g.qk);
  c.rc2q = ldexpf(c.rc2f, 2 * g.qk);
  c.c2q = ldexpf(c.c2f, -2 * g.qk);

  // FP32 list filter on hi parts: each hi difference is exact and differs from the exact
  // difference by at most eps = 2^(p-22) + 2^(p-24) (two dropped lo parts, the split of L and
  // the rounding of an image shift of hi that leaves its binade), so
  // |r2f - r^2| <= eps (2 sqrt(3) r_s + 3 eps) + 4 ulp(r_s^2).  Twice that bound plus 1e-6
  // relative is the band around r_s^2 inside which the exact FP64 test decides.
  {
    const double eps = ldexp(1.0, pw - 22) + ldexp(1.0, pw - 24);
    const double bound = eps * (2.0 * sqrt(3.0) * rs + 3.0 * eps) + 4.0 * 1.2e-7 * rs * rs;
    const double band = 2.0 * bound + 1e-6 * rs * rs;
    s->band.rs2 = rs * rs;
    s->band.lo = (float)(rs * rs - band);
    s->band.hi = (float)(rs * rs + band);
  }
  // Displacement rule: rebuild when max |x - x_ref| > margin / 2.  The mixed form measures it on
  // the fixed-point records (each component within u of the FP64 difference, then FP32 rounding),
  // so the limit is lowered by twice that bound and a relative 2e-6 of margin/2; the FP64 form
  // rounds the squared displacement up.
  s->disp_limit = 0.5 * p.margin - disp_slack(s);
  return LJ_OK;
}

// The list form in use.  LJ_LIST_AUTO takes the half list in the FP64 form (its pair arithmetic
// runs on the FP64 pipe, so halving the pairs pays for the atomics) and, in the mixed form, when
// the full list would hold 75 or more partners per particle, (4/3) pi r_s^3 N / L^3: the crossover
// measured on GB300 at 16.4M particles (full list faster at 56 partners, rho = 0.5; half list
// faster at 87, rho = 0.8).  A change of form invalidates the list.
static void resolve_list_form(ljmd_sys* s) {
  bool half = s->prm.list_form == LJ_LIST_HALF;
  if (s->prm.list_form == LJ_LIST_AUTO) {
    const double per = 4.18879020478639 * s->rs * s->rs * s->rs * (double)s->n / (s->L * s->L * s->L);
    half = s->precision != LJ_MIXED || per >= 75.0;
  }
  if (half != s->list_half) {
    s->list_half = half;
    s->have_list = false;
    s->forces_current = false;
  }
}

// The adjoint kernel writes each key's Hessian-vector row from the key's own list row, so it
// needs the full list.  An explicit half list is refused (LJ_ESTATE); LJ_LIST_AUTO is fixed to the
// full list from then on.
static int adjoint_list_form(ljmd_sys* s) {
  if (s->prm.list_form == LJ_LIST_HALF) return LJ_ESTATE;
  if (s->prm.list_form == LJ_LIST_AUTO) {
    s->prm.list_form = LJ_LIST_FULL;
    resolve_list_form(s);
  }
  return LJ_OK;
}

static int ensure_particles(ljmd_sys* s, int64_t n) {
  if (n <= s->cap_n) return LJ_OK;
  const bool mixed = s->precision == LJ_MIXED;
  const size_t fsz = mixed ? sizeof(float4) : sizeof(dvec4);
  TRY(dalloc_t(s, &s->x, 3 * n));
  TRY(dalloc_t(s, &s->v, 3 * n));
  TRY(dalloc_t(s, &s->x_alt, 3 * n));
  TRY(dalloc_t(s, &s->v_alt, 3 * n));
  TRY(dalloc(s, &s->f, fsz * n));
  TRY(dalloc(s, &s->f_alt, fsz * n));
  TRY(dalloc_t(s, &s->hi, n));
  if (mixed) TRY(dalloc_t(s, &s->xq, n));
  if (!mixed) TRY(dalloc_t(s, &s->pos64, n));
  TRY(dalloc(s, &s->ref, fsz * n));
  TRY(dalloc_t(s, &s->id, n));
  TRY(dalloc_t(s, &s->id_alt, n));
  TRY(dalloc_t(s, &s->img, 3 * n));
  TRY(dalloc_t(s, &s->img_alt, 3 * n));
  TRY(dalloc_t(s, &s->cell_of, n));
  TRY(dalloc_t(s, &s->perm, n));
  TRY(dalloc_t(s, &s->perm_id, n));
  TRY(dalloc_t(s, &s->rows, n + 2));  // +2: aligned bulk copies of a tile's rows may read past the end
  s->cap_n = n;
  return LJ_OK;
}

static int ensure_scan_tmp(ljmd_sys* s, int64_t n) {
  const size_t w = scan_tmp_words(n);
  if (w <= s->scan_tmp_cap) return LJ_OK;
  TRY(dalloc_t(s, &s->scan_tmp, w));
  s->scan_tmp_cap = w;
  return LJ_OK;
}

static int ensure_cells(ljmd_sys* s) {
  if (s->ncells > s->cap_cells) {
    TRY(dalloc_t(s, &s->cell_count, s->ncells));
    TRY(dalloc_t(s, &s->cell_start, s->ncells + 1));
    TRY(dalloc_t(s, &s->cell_fill, s->ncells));
    s->cap_cells = s->ncells;
  }
  TRY(ensure_scan_tmp(s, s->ncells));
  TRY(ensure_scan_tmp(s, s->n));
  return LJ_OK;
}

static void reset_counters(ljmd_sys* s) {
  s->last_build_step = 0;
  s->lifetime_est = 16;
  s->ldc_checks = 0;
  s->ldc_kept = 0;
  s->have_list = false;
  s->forces_current = false;
  s->pe_step = -1;
  s->energy_step = -1;
  s->steps = 0;
  s->rebuilds = 0;
  s->list_entries = 0;
  s->last_dmax = 0.0;
}

static int device_status(ljmd_sys* s, int32_t* out) {
  ljmd_sys* sys = s;
  CK(cudaMemcpyAsync(s->h_i32, s->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  *out = *s->h_i32;
  return LJ_OK;
}

static int check_status(ljmd_sys* s) {
  int32_t w = 0;
  TRY(device_status(s, &w));
  return w ? LJ_EDEVICE : LJ_OK;
}

static void* force_pos(ljmd_sys* s);

static int ensure_tile_list(ljmd_sys* s) {
  if (s->ta.ntiles > s->tile_list_cap) {
    TRY(dalloc_t(s, &s->tile_list, s->ta.ntiles));
    s->tile_list_cap = s->ta.ntiles;
  }
  return LJ_OK;
}

// Tile geometry for the staged list/force kernels: T cells along z per tile, shared-memory
// capacities from the actual largest tile of the current cell occupancy.
// Tile buffers per force CTA: the requested number, else two for the forms with a pipelined
// kernel (producer warps stage the next tile while consumer warps compute): the mixed form with
// the full list and the FP64 form with the half list; one otherwise.
// Multiprocessors of a device (152 if the attribute cannot be read).
static int sm_count_of(int dev) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
    cudaGetLastError();
    sms = 152;
  }
  return sms;
}

static int force_buffers(const ljmd_sys* s) {
  if (s->force_nbuf) return s->force_nbuf;
  // fewer tiles than two per SM: the single-buffer kernel (the pipelined one holds one CTA per SM
  // with two producer warps; 4,000 particles, FP64 form: 40 against 44 us per force launch)
  if (s->ta.ntiles > 0 && s->ta.ntiles < 2 * (int64_t)sm_count_of(s->device)) return 1;
  return ((s->precision == LJ_MIXED) != s->list_half) ? 2 : 1;
}

// Default cells per tile along z.  The mixed form with the full list (the pipelined force kernel):
// about 165 key particles per tile, so that the staging of the 9 (T + 2) neighbour cells and the
// per-tile bookkeeping are spread over many keys; measured on GB300 at 16.4M particles, rho 0.5
// (13.8 particles per cell), T = 4, 8, 10, 12 give force launches of 2.41, 2.09, 1.96, 1.88 ms and
// list constructions of 11.7, 14.0, 13.2, 13.2 ms, and T = 12 the shortest step.  The half-list
// forms keep 4 cells: at rho 0.8 (mixed, half list) T = 3, 4, 6 give force 3.76, 3.56, 4.06 ms and
// construction 19.0, 19.8, 33.7 ms; the FP64 form at rho 0.5 gives force 45.5 ms at T = 4 and
// 49.4 ms at T = 10 with 2 lanes.
// Small boxes: the tile length is lowered until there are at least two tiles per SM, so that the
// force launch spreads over the GPU (4,000 particles, 6 cells per side, FP64 form: T = 4, 2, 1 give
// 72, 108, 216 tiles and force launches of 69, 40, 39 us).
static int default_tile_cells(const ljmd_sys* s) {
  int T = 4;
  if (s->precision == LJ_MIXED && !s->list_half) {
    const double ppc = (double)s->n / (double)std::max<int64_t>(s->ncells, 1);
    T = std::max(1, std::min((int)lround(165.0 / std::max(ppc, 1.0)), 12));
  }
  const int64_t n = s->g.n, want = 2 * (int64_t)sm_count_of(s->device);
  while (T > 1 && n * n * ((n + T - 1) / T) < want) --T;
  return T;
}

// Default threads per key in the force kernel: for the mixed form with the full list, 2 for tiles
// of about 100 keys or more (more keys than 4-lane groups otherwise), 4 below (measured as above:
// T = 10 with 2 lanes 1.96 ms, 4 lanes 2.01 ms; T = 4 with 2 lanes 2.41 ms, 4 lanes 2.41 ms,
// 8 lanes 2.67 ms); 4 for the half-list forms.
static int default_lanes(const ljmd_sys* s) {
  const double ppc = (double)s->n / (double)std::max<int64_t>(s->ncells, 1);
  if (s->precision != LJ_MIXED || s->list_half) return (double)s->ta.T * ppc <= 32.0 ? 8 : 4;
  return (double)s->ta.T * ppc >= 96.0 ? 2 : 4;
}

static int choose_tiles(ljmd_sys* s, int t_cap) {
  ljmd_sys* sys = s;
  TileArgs& ta = s->ta;
  const int n = s->g.n;
  ta.n = n;
  int dev = 0, smem_max = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (n < 3) {
    ta.whole = 1;
    ta.T = 1;
    ta.ntz = 1;
    ta.ntiles = 1;
    ta.max_staged = (int32_t)s->n;
    ta.max_own = (int32_t)s->n;
    ta.max_chunks = (int32_t)((s->n + 31) / 32);
    if (s->n > 65535 || list_smem_bytes(ta, s->precision) > (size_t)smem_max) return LJ_ERANGE;
    return ensure_tile_list(s);
  }
  ta.whole = 0;
  int T = s->tile_T > 0 ? s->tile_T : default_tile_cells(s);
  if (T > t_cap) T = t_cap;
  if (T > n - 2) T = n - 2;
  if (T > kMaxTileT) T = kMaxTileT;
  if (T < 1) T = 1;
  for (;; --T) {
    ta.T = T;
    ta.ntz = (n + T - 1) / T;
    ta.ntiles = (int64_t)n * n * ta.ntz;
    CK(cudaMemsetAsync(s->d_sizes, 0, 3 * sizeof(unsigned int), s->st));
    launch_tile_sizes(s->cell_start, ta, s->d_sizes, s->st);
    launch_max_count(s->cell_count, s->ncells, s->d_sizes + 2, s->st);
    s->launches += 2;
    CKL();
    CK(cudaMemcpyAsync(s->h_u32 + 8, s->d_sizes, 3 * sizeof(unsigned int), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    const unsigned staged = s->h_u32[8], own = s->h_u32[9], maxcell = s->h_u32[10];
    ta.max_staged = (int32_t)staged;
    ta.max_own = (int32_t)(own > 0 ? own : 1);
    ta.max_chunks = (int32_t)(9 * ((3 * maxcell + 31) / 32) + 1);
    if (staged <= 65535 && list_smem_bytes(ta, s->precision) <= (size_t)smem_max) return ensure_tile_list(s);
    if (T == 1) return LJ_ERANGE;  // cell occupancy beyond what a tile can stage
  }
}

// ----------------------------------------------------------------------------------------------
// Pair-list construction: fold, label, counting sort (Fig. 3), reorder (Sec. 3.3), sorted list.
static int rebuild(ljmd_sys* s) {
  ljmd_sys* sys = s;
  const int64_t N = s->n;
  cudaStream_t st = s->st;
  TRY(ensure_cells(s));
  PhaseTimer timer(s, PH_REBUILD);
  // wrap_label, scatter, cell_order, gather, shadow (+ the scan, tile sizing and list below)
  s->launches += 5;
  CK(cudaMemsetAsync(s->cell_count, 0, sizeof(uint32_t) * s->ncells, st));
  launch_wrap_label(s->x, s->img, N, s->g, s->cell_of, s->cell_count, s->d_status, st);
  CKL();
  s->launches += launch_scan_u32(s->cell_count, s->cell_start, s->ncells, s->scan_tmp, st);
  CKL();
  CK(cudaMemsetAsync(s->cell_fill, 0, sizeof(uint32_t) * s->ncells, st));
  launch_scatter(s->cell_of, s->cell_start, s->cell_fill, s->perm, N, st);
  launch_cell_rank(s->cell_start, s->ncells, s->perm, s->id, s->perm_id, st);
  launch_gather_state(s->perm_id, N, s->x, s->x_alt, s->v, s->v_alt, s->id, s->id_alt, s->img, s->img_alt, s->f,
                      s->f_alt, s->precision == LJ_MIXED ? 16 : 32, st, nullptr);
  CKL();
  std::swap(s->x, s->x_alt);
  std::swap(s->v, s->v_alt);
  std::swap(s->id, s->id_alt);
  std::swap(s->img, s->img_alt);
  std::swap(s->f, s->f_alt);
  launch_shadow_all(s->x, N, s->precision == LJ_MIXED, s->g.qk, s->hi, s->xq, s->pos64, s->ref, st);
  CKL();
  const int half = s->list_half ? 1 : 0;
  uint64_t total = 0;
  int dev = 0, smem_max = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // the force kernel's two tile buffers must fit: a smaller tile is chosen if they do not
  for (int t_cap = kMaxTileT;;) {
    TRY(choose_tiles(s, t_cap));
    bool built = false;
    for (int attempt = 0; attempt < 2; ++attempt) {
      if (s->ent_cap == 0) {
        // first construction: the continuum estimate of partners within r_s, with headroom
        const double est = 4.18879 * s->rs * s->rs * s->rs * (double)N / (s->L * s->L * s->L);
        const size_t want = (size_t)((double)N * (est * (half ? 0.5 : 1.0) * 1.3 + 8.0)) + 4096;
        TRY(dalloc_t(s, &s->ent, want));
        s->ent_cap = want;
      }
      CK(cudaMemsetAsync(s->d_total64, 0, 2 * sizeof(unsigned long long), st));
      CK(cudaMemsetAsync(s->d_sizes + 3, 0, sizeof(unsigned int), st));
      // the list kernels filter on the FP32 hi copies (mixed) or the FP64 copies (FP64 form, whole box)
      const void* list_pos = s->precision == LJ_MIXED ? (const void*)s->hi : (const void*)s->pos64;
      launch_list_tile(s->precision, half, list_pos, s->hi, s->x, s->cell_start, N, s->g, s->ta, s->band, s->rows,
                       s->tile_list, s->ent, (uint64_t)s->ent_cap, s->d_total64, s->d_sizes + 3, s->d_status, st);
      s->launches += 1;
      CKL();
      CK(cudaMemcpyAsync(s->h_u32 + 4, s->d_total64, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(s->h_u32 + 12, s->d_sizes + 3, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(s->h_u32 + 13, s->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));  // one round trip: list size, longest segment and status
      unsigned long long total64, actual64;
      memcpy(&total64, s->h_u32 + 4, sizeof(total64));
      memcpy(&actual64, s->h_u32 + 6, sizeof(actual64));
      s->ta.max_list = (int32_t)s->h_u32[12];
      if (total64 > 4294967295ULL) return LJ_ERANGE;  // row starts are 32-bit
      total = total64;
      if (total <= s->ent_cap) {
        int32_t w = 0;
        memcpy(&w, s->h_u32 + 13, sizeof(w));
        if (w) {
          fprintf(stderr, "ljmd: list construction raised status %d (n=%d T=%d tiles=%lld staged<=%d own<=%d)\n", w,
                  s->ta.n, s->ta.T, (long long)s->ta.ntiles, s->ta.max_staged, s->ta.max_own);
          return LJ_EDEVICE;
        }
        s->list_actual = actual64;
        built = true;
        break;
      }
      // the rows did not fit: grow to the exact size plus headroom and construct again
      const size_t want = (size_t)(total * 1.2) + 4096;
      TRY(dalloc_t(s, &s->ent, want));
      s->ent_cap = want;
    }
    if (!built) return LJ_EDEVICE;
    // the force kernel stages a tile's list segment if it fits; longer segments are read from HBM
    TileArgs tz = s->ta;
    tz.list_cap = 0;
    const size_t base_bytes = std::max(force_smem_bytes(tz, s->precision, force_buffers(s), 1),
                                       adjoint_smem_bytes(tz, s->precision));
    const int nbuf = s->ta.whole ? 1 : force_buffers(s);
    if (base_bytes <= (size_t)smem_max) {
      int64_t room = ((int64_t)smem_max - (int64_t)base_bytes) / (2 * nbuf) - 16;
      // The pipelined kernel of the mixed form with the full list runs 3 CTAs per SM with 8
      // consumer warps (T <= 4) and 2 with 12: the staged segments are capped so that this many
      // fit in an SM's shared memory (1 KB reserved and at most 6 KB of static shared memory per
      // CTA), when that still stages at least half of the largest segment.  Longer segments are
      // read from HBM (on the FCC start, whose longest segment is 1.5 times the liquid's, this
      // still beat one CTA per SM: 16.4M, 20 steps, 3.41 -> 3.35 ms per step).
      if (s->precision == LJ_MIXED && !s->list_half && !s->ta.whole && nbuf == 2) {
        int smem_sm = 0;
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        const int target = s->ta.T <= 4 ? 3 : 2;
        const int64_t per_cta = (int64_t)smem_sm / target - 1024 - 6144;
        const int64_t fb = (int64_t)force_smem_bytes(tz, s->precision, 2, 0);
        const int64_t room_occ = (per_cta - fb) / (2 * nbuf) - 16;
        if (room_occ >= (int64_t)s->ta.max_list / 2) room = std::min(room, room_occ);
      }
      s->ta.list_cap = (int32_t)std::max<int64_t>(0, std::min<int64_t>(s->ta.max_list, room) & ~(int64_t)7);
      break;
    }
    if (s->ta.whole || s->ta.T <= 1) return LJ_ERANGE;
    t_cap = s->ta.T - 1;
  }
  s->list_entries = total;
  s->have_list = true;
  if (s->rebuilds > 0 && s->steps > s->last_build_step) s->lifetime_est = s->steps - s->last_build_step;
  s->last_build_step = s->steps;
  s->rebuilds += 1;
  s->dutc_buffer = s->prm.margin;
  if (s->valid_mode == LJ_VALID_DUTC_LDC || s->valid_mode == LJ_VALID_HALF_MARGIN_LDC) {
    if (s->xref_cap < s->n) {
      TRY(dalloc_t(s, &s->xref64, 3 * (size_t)s->n));
      s->xref_cap = s->n;
    }
    launch_copy_words(s->x, s->xref64, 24 * s->n, nullptr, s->st);
    s->launches += 1;
  }
  s->pe_step = -1;
  return LJ_OK;
}

static void* force_pos(ljmd_sys* s) { return s->precision == LJ_MIXED ? (void*)s->xq : (void*)s->pos64; }

static int integrate(ljmd_sys* s, IntegrateArgs a, const int* skip = nullptr, const StepFinish* fin = nullptr) {
  PhaseTimer timer(s, PH_INTEGRATE);
  s->launches += 1;
  a.qk = s->g.qk;
  return launch_integrate(s->precision, s->x, s->v, s->f, force_pos(s), s->ref, s->n, a, s->part_ke, s->d_dmax,
                          s->d_status, fin ? *fin : StepFinish{}, s->st, skip);
}

// Energy record of state `step` (default: the current one); skipped on the device if *skip is set.
static void energy_record(ljmd_sys* s, int nb_ke, bool to_log, int64_t step = -1, const int* skip = nullptr) {
  PhaseTimer timer(s, PH_ENERGY);
  s->launches += 1;
  if (step < 0) step = s->steps;
  const double scale = s->list_half ? 1.0 : 0.5;
  launch_energy_finalize(s->part_force, s->nb_force, s->part_ke, nb_ke, scale, s->d_energies,
                         to_log ? s->log_ptr : nullptr, to_log ? s->log_cap : 0, s->d_log_count, (double)step, s->st,
                         skip);
  s->energy_step = step;
}

static int run_force(ljmd_sys* s, bool energy, const int* skip = nullptr) {
  ljmd_sys* sys = s;
  const int half = s->list_half ? 1 : 0;
  if (half) CK(cudaMemsetAsync(s->f, 0, (s->precision == LJ_MIXED ? 16 : 32) * (size_t)s->n, s->st));
  int lanes = s->prm.lanes;
  if (lanes == 0) lanes = default_lanes(s);
  const int per_sm = s->force_per_sm;  // 0: as many CTAs per SM as shared memory allows
  {
    PhaseTimer timer(s, PH_FORCE);
    s->nb_force = launch_force_tile(s->precision, half, lanes, energy ? 1 : 0, force_pos(s), s->cell_start, s->n, s->g,
                                    s->ta, s->c, s->rows, s->tile_list, s->ent, s->f, s->part_force, s->d_status,
                                    per_sm, force_buffers(s), s->st, skip);
  }
  s->launches += 1;
  CKL();
  s->forces_current = true;
  s->pe_step = energy ? s->steps : -1;
  return LJ_OK;
}

// Largest displacement since the list was built, as measured by the last integrate launch.
static int read_dmax(ljmd_sys* s, double* out) {
  ljmd_sys* sys = s;
  CK(cudaMemcpyAsync(s->h_u32, s->d_dmax, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  float d2, v2;
  memcpy(&d2, s->h_u32, sizeof(float));
  memcpy(&v2, s->h_u32 + 1, sizeof(float));
  *out = sqrt((double)d2);
  s->last_vmax = sqrt((double)v2);
  return LJ_OK;
}

// Large displacement check (Alg. 2): L_D = particles that moved more than margin - d_max (d_max
// taken as an upper bound of the measured largest displacement); the list stays valid if |L_D| <=
// N_l and no pair of L_D is both unlisted and now closer than r_c.  Synchronises twice.
static int ldc_valid(ljmd_sys* s, bool* valid) {
  ljmd_sys* sys = s;
  *valid = false;
  s->ldc_checks += 1;
  const double th = s->prm.margin - (s->last_dmax + disp_slack(s)) - 1e-9;
  if (!(th > 0.0) || !s->xref64) return LJ_OK;
  if (!s->ldc_list) TRY(dalloc_t(s, &s->ldc_list, (size_t)s->max_ld));
  if (!s->d_ldc) TRY(dalloc_t(s, &s->d_ldc, 2));
  CK(cudaMemsetAsync(s->d_ldc, 0, 2 * sizeof(unsigned int), s->st));
  launch_ldc_collect(s->x, s->xref64, s->n, th * th, s->ldc_list, (unsigned)s->max_ld, s->d_ldc, s->st);
  s->launches += 1;
  CKL();
  CK(cudaMemcpyAsync(s->h_u32, s->d_ldc, sizeof(unsigned int), cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  const unsigned int m = s->h_u32[0];
  if (m > (unsigned)s->max_ld) return LJ_OK;
  if (m >= 2) {
    launch_ldc_pairs(s->x, s->xref64, s->n, s->g, s->ldc_list, (int)m, s->band.rs2, s->c.rc2, (int*)s->d_ldc + 1,
                     s->st);
    s->launches += 1;
    CKL();
    CK(cudaMemcpyAsync(s->h_u32, s->d_ldc + 1, sizeof(unsigned int), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    if (s->h_u32[0]) return LJ_OK;
  }
  *valid = true;
  s->ldc_kept += 1;
  return LJ_OK;
}

// The list-validity rule after a drift of length dt (measured maxima of the step are current).
static int list_expired(ljmd_sys* s, double dt, bool* expired) {
  *expired = false;
  switch (s->valid_mode) {
    case LJ_VALID_HALF_MARGIN:
      *expired = s->last_dmax > s->disp_limit;
      return LJ_OK;
    case LJ_VALID_DUTC:
      s->dutc_buffer -= 2.0 * s->last_vmax * (1.0 + 1e-6) * fabs(dt);
      *expired = !(s->dutc_buffer > 0.0);
      return LJ_OK;
    default: {
      bool first_ok;
      if (s->valid_mode == LJ_VALID_DUTC_LDC) {
        s->dutc_buffer -= 2.0 * s->last_vmax * (1.0 + 1e-6) * fabs(dt);
        first_ok = s->dutc_buffer > 0.0;
      } else {
        first_ok = s->last_dmax <= s->disp_limit;
      }
      if (first_ok) return LJ_OK;
      bool ok = false;
      TRY(ldc_valid(s, &ok));
      *expired = !ok;
      return LJ_OK;
    }
  }
}

static int ensure_forces(ljmd_sys* s, bool energy) {
  if (!s->have_list) TRY(rebuild(s));
  if (!s->forces_current || (energy && s->pe_step != s->steps)) TRY(run_force(s, energy));
  return LJ_OK;
}

// KE of the current (full-step) velocities and the energy record of the current state.
static int finalize_energies_now(ljmd_sys* s) {
  ljmd_sys* sys = s;
  TRY(ensure_forces(s, true));
  IntegrateArgs a{0.0, 0.0, 0.0, 1, 0};
  const int nb = integrate(s, a);
  CKL();
  energy_record(s, nb, false);
  CKL();
  return LJ_OK;
}

// Up to `remaining` velocity-Verlet steps with the list-validity rule decided on the device: each
// step is the kick-drift (with the first half-kick fused into the previous step's second, except
// for the first step of the call), whose last CTA takes the energy record when due and the validity
// check, and the force; all of them are enqueued at once and the host synchronises once at the end.  When
// the check of a step finds the list expired it sets the stop flag, which every later launch of
// the run reads first and returns on; that step's drift has happened but not its force.  The run
// is sized from the lifetime of the last list, so that few launches are skipped.  *advanced: the
// steps whose drift happened; *stopped: the last of them expired the list.
static int device_run(ljmd_sys* s, double dt, bool first_of_call, int64_t remaining, int64_t* advanced,
                      bool* stopped) {
  ljmd_sys* sys = s;
  cudaStream_t st = s->st;
  const int ee = s->prm.energy_every;
  auto want_energy = [&](int64_t t) { return ee > 0 && (t % ee) == 0; };
  const double h = 0.5 * dt;
  const int dutc = s->valid_mode == LJ_VALID_DUTC;
  const int64_t age = s->steps - s->last_build_step;
  const int64_t K = std::max<int64_t>(1, std::min<int64_t>({remaining, std::max<int64_t>(4, s->lifetime_est - age + 2),
                                                           256}));
  StepCtl* hc = s->h_ctl;
  hc->stop = 0;
  hc->stop_at = -1;
  hc->last[0] = hc->last[1] = 0.0f;
  hc->dutc = s->dutc_buffer;
  CK(cudaMemcpyAsync(s->d_ctl, hc, sizeof(StepCtl), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(s->d_dmax, 0, 8, st));
  const int* skip = &s->d_ctl->stop;
  const size_t ev0 = s->ev_pending.size();
  const int64_t energy_step0 = s->energy_step;
  std::vector<size_t> ev_force(K);     // profiling entries before each step's force launch
  std::vector<int64_t> ln_force(K);    // launch count before each step's force launch
  std::vector<char> recorded(K, 0);
  for (int64_t k = 0; k < K; ++k) {
    const int64_t t = s->steps + k;  // state index before the step
    const bool rec = (k == 0 ? s->pe_step == s->steps : true) && want_energy(t);
    IntegrateArgs a{(first_of_call && k == 0) ? 0.0 : h, h, dt, rec ? 1 : 0, 1, dutc};
    // the integrator's last CTA records the energies of state t and takes the validity check
    StepFinish fin{};
    fin.ticket = s->d_ticket;
    fin.rec = rec ? 1 : 0;
    fin.pv = s->part_force;
    fin.nbf = s->nb_force;
    fin.pe_scale = s->list_half ? 1.0 : 0.5;
    fin.energies = s->d_energies;
    fin.log = s->log_ptr;
    fin.cap = s->log_cap;
    fin.count = s->d_log_count;
    fin.step = (double)t;
    fin.check = 1;
    fin.ctl = s->d_ctl;
    fin.s = (int)k;
    fin.disp_limit = s->disp_limit;
    fin.dutc = dutc;
    fin.two_dt = 2.0 * fabs(dt);
    integrate(s, a, skip, &fin);
    if (rec) recorded[k] = 1;
    if (s->cap_x) {  // the state after this step's drift (skipped if the run stopped earlier)
      launch_unwrapped(s->x, s->img, s->id, s->n, s->g.offset, s->L, s->cap_x + 3 * s->n * (t + 1 - s->cap_step0),
                       st, s->d_ctl, (int)k);
      s->launches += 1;
    }
    ev_force[k] = s->ev_pending.size();
    ln_force[k] = s->launches;
    TRY(run_force(s, want_energy(t + 1), skip));
  }
  CKL();
  CK(cudaMemcpyAsync(hc, s->d_ctl, sizeof(StepCtl), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  *stopped = hc->stop != 0;
  const int64_t done = *stopped ? (int64_t)hc->stop_at + 1 : K;
  // skipped launches of the run leave the counters and the profile; the stopping step's force too
  if (*stopped && s->profiling && ev_force[done - 1] >= ev0 && ev_force[done - 1] <= s->ev_pending.size()) {
    for (size_t q = ev_force[done - 1]; q < s->ev_pending.size(); ++q) {
      s->ev_pool.push_back(s->ev_pending[q].second.first);
      s->ev_pool.push_back(s->ev_pending[q].second.second);
    }
    s->ev_pending.resize(ev_force[done - 1]);
  }
  if (*stopped) s->launches = ln_force[done - 1];  // launches that ran: up to the stopping step's check
  s->energy_step = energy_step0;
  for (int64_t k = 0; k < done; ++k)
    if (recorded[k]) s->energy_step = s->steps + k;
  s->steps += done;
  *advanced = done;
  s->last_dmax = sqrt((double)hc->last[0]);
  s->last_vmax = sqrt((double)hc->last[1]);
  s->dutc_buffer = hc->dutc;
  if (*stopped) {
    s->forces_current = false;
    s->pe_step = -1;
  } else {
    s->forces_current = true;
    s->pe_step = want_energy(s->steps) ? s->steps : -1;
  }
  return LJ_OK;
}

static int step_steps(ljmd_sys* sys, double dt, int64_t nsteps);

// ----------------------------------------------------------------------------------------------
extern "C" {

int ljmd_version(void) { return 100; }

const char* ljmd_strerror(int code) {
  switch (code) {
    case LJ_OK: return "ok";
    case LJ_EINVAL: return "invalid argument";
    case LJ_ENOMEM: return "out of memory";
    case LJ_EDEVICE: return "CUDA error or device status raised";
    case LJ_ESTATE: return "call out of order (no particles)";
    case LJ_ERANGE: return "size beyond a library limit";
    default: return "unknown status";
  }
}

int ljmd_create(ljmd_sys** out, const ljmd_params* p, int32_t precision, void* cuda_stream) {
  if (!out || !p) return LJ_EINVAL;
  *out = nullptr;
  if (precision != LJ_FP64 && precision != LJ_MIXED) return LJ_EINVAL;
  if (check_params(p) != LJ_OK) return LJ_EINVAL;
  ljmd_sys* sys = new (std::nothrow) ljmd_sys();
  if (!sys) return LJ_ENOMEM;
  sys->prm = *p;
  sys->precision = precision;
  sys->st = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&sys->device) != cudaSuccess) {
    cudaGetLastError();
    delete sys;
    return LJ_EDEVICE;
  }
  int r = LJ_OK;
  if (r == LJ_OK) r = dalloc_t(sys, &sys->part_force, 2 * kMaxRedBlocks);
  if (r == LJ_OK) r = dalloc_t(sys, &sys->part_ke, kMaxRedBlocks);
  if (r == LJ_OK) r = dalloc_t(sys, &sys->part_misc, 4 * kMaxRedBlocks);
  if (r == LJ_OK) r = dalloc_t(sys, &sys->d_scalars, 8);
  if (r == LJ_OK) r = dalloc_t(sys, &sys->d_energies, 4);
  if (r == LJ_OK) r = dalloc_t(sys, &sys->d_log_count, 1);
  if (r == LJ_OK) r = dalloc_t(sys, &sys->d_status, 1);
  if (r == LJ_OK) r = dalloc_t(sys, &sys->d_dmax, 2);
  if (r == LJ_OK) r = dalloc_t(sys, &sys->d_ctl, 1);
  if (r == LJ_OK) r = dalloc_t(sys, &sys->d_ticket, 1);
  if (r == LJ_OK && cudaMemsetAsync(sys->d_ticket, 0, sizeof(unsigned int), sys->st) != cudaSuccess) r = LJ_EDEVICE;
  if (r == LJ_OK && cudaMallocHost(&sys->h_ctl, sizeof(StepCtl)) != cudaSuccess) r = LJ_ENOMEM;
  if (r == LJ_OK) r = dalloc_t(sys, &sys->d_total64, 2);
  if (r == LJ_OK) r = dalloc_t(sys, &sys->d_sizes, 4);
  if (r == LJ_OK && cudaMallocHost(&sys->h_u32, 64) != cudaSuccess) r = LJ_ENOMEM;
  if (r == LJ_OK && cudaMallocHost(&sys->h_f64, 64) != cudaSuccess) r = LJ_ENOMEM;
  if (r == LJ_OK && cudaMallocHost(&sys->h_i32, 64) != cudaSuccess) r = LJ_ENOMEM;
  if (r == LJ_OK && cudaMemsetAsync(sys->d_status, 0, 4, sys->st) != cudaSuccess) r = LJ_EDEVICE;
  if (r == LJ_OK && cudaMemsetAsync(sys->d_log_count, 0, 8, sys->st) != cudaSuccess) r = LJ_EDEVICE;
  if (r != LJ_OK) {
    cudaGetLastError();
    free_all(sys);
    delete sys;
    return r;
  }
  *out = sys;
  return LJ_OK;
}

void ljmd_destroy(ljmd_sys* sys) {
  if (!sys) return;
  if (sys->st) cudaStreamSynchronize(sys->st);
  else cudaDeviceSynchronize();
  free_all(sys);
  cudaGetLastError();
  delete sys;
}

int ljmd_init_lattice(ljmd_sys* sys, int64_t M, double density, double T, uint64_t seed) {
  if (!sys || M <= 0 || !(density > 0.0) || !(T >= 0.0)) return LJ_EINVAL;
  if (sys->broken) return LJ_EDEVICE;
  if (M > 2000) return LJ_ERANGE;
  const int64_t N = 4 * M * M * M;
  if (N > 1000000000LL) return LJ_ERANGE;
  const double a = cbrt(4.0 / density);
  TRY(setup_geometry(sys, a * (double)M));
  TRY(ensure_particles(sys, N));
  sys->n = N;
  resolve_list_form(sys);
  TRY(ensure_cells(sys));
  reset_counters(sys);
  launch_fcc(sys->x, M, a, sys->g.offset, sys->st);
  CKL();
  launch_gaussian(sys->v, N, seed, sys->st);
  CKL();
  const int nb = red_blocks(N);
  launch_sums3(sys->v, N, sys->part_misc, nb, sys->st);
  launch_final_reduce(sys->part_misc, nb, 3, sys->d_scalars, sys->st);
  launch_sumsq_centered(sys->v, N, sys->d_scalars, sys->part_misc, nb, sys->st);
  launch_final_reduce(sys->part_misc, nb, 1, sys->d_scalars + 4, sys->st);
  launch_center_scale(sys->v, N, sys->d_scalars, sys->d_scalars + 4, T, sys->st);
  CKL();
  CK(cudaMemsetAsync(sys->img, 0, sizeof(int32_t) * 3 * N, sys->st));
  CK(cudaMemsetAsync(sys->f, 0, (sys->precision == LJ_MIXED ? 16 : 32) * (size_t)N, sys->st));
  launch_iota_i32(sys->id, N, sys->st);  // id = lattice order
  CKL();
  return LJ_OK;
}

int ljmd_set_state(ljmd_sys* sys, int64_t n, double box, const double* x, const double* v, int32_t on_device) {
  if (!sys || n <= 0 || !x) return LJ_EINVAL;
  if (sys->broken) return LJ_EDEVICE;
  if (n > 1000000000LL) return LJ_ERANGE;
  TRY(setup_geometry(sys, box));
  TRY(ensure_particles(sys, n));
  sys->n = n;
  resolve_list_form(sys);
  TRY(ensure_cells(sys));
  reset_counters(sys);
  const double* xs = x;
  const double* vs = v;
  if (!on_device) {
    CK(cudaMemcpyAsync(sys->x_alt, x, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, sys->st));
    xs = sys->x_alt;
    if (v) {
      CK(cudaMemcpyAsync(sys->v_alt, v, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, sys->st));
      vs = sys->v_alt;
    }
  }
  launch_load_state(xs, vs, sys->x, sys->v, sys->id, sys->img, n, sys->g.offset, sys->L, sys->st);
  CKL();
  CK(cudaMemsetAsync(sys->f, 0, (sys->precision == LJ_MIXED ? 16 : 32) * (size_t)n, sys->st));
  if (!on_device) CK(cudaStreamSynchronize(sys->st));  // host buffers may be reused by the caller
  return LJ_OK;
}

int ljmd_get_state(ljmd_sys* sys, double* x, double* v, double* f, int32_t* img, int32_t on_device) {
  if (!sys) return LJ_EINVAL;
  if (sys->broken) return LJ_EDEVICE;
  if (sys->n <= 0) return LJ_ESTATE;
  const int64_t N = sys->n;
  cudaStream_t st = sys->st;
  // x_alt / v_alt / img_alt are free between list constructions and serve as staging
  if (x) {
    double* dst = on_device ? x : sys->x_alt;
    launch_scatter_back_f64x3(sys->x, dst, sys->id, N, sys->g.offset, st);
    CKL();
    if (!on_device) CK(cudaMemcpyAsync(x, dst, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, st));
  }
  if (v) {
    double* dst = on_device ? v : sys->v_alt;
    launch_scatter_back_f64x3(sys->v, dst, sys->id, N, 0.0, st);
    CKL();
    if (!on_device) CK(cudaMemcpyAsync(v, dst, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, st));
  }
  if (f) {
    CK(cudaStreamSynchronize(st));  // x_alt may be in use by the x copy above
    double* dst = on_device ? f : sys->x_alt;
    if (sys->precision == LJ_MIXED) launch_scatter_back_f32x4_to_f64x3((const float4*)sys->f, dst, sys->id, N, st);
    else launch_scatter_back_f64x4_to_f64x3((const dvec4*)sys->f, dst, sys->id, N, st);
    CKL();
    if (!on_device) CK(cudaMemcpyAsync(f, dst, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, st));
  }
  if (img) {
    int32_t* dst = on_device ? img : sys->img_alt;
    launch_scatter_back_i32x3(sys->img, dst, sys->id, N, st);
    CKL();
    if (!on_device) CK(cudaMemcpyAsync(img, dst, sizeof(int32_t) * 3 * N, cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  return check_status(sys);
}

int ljmd_build_pairlist(ljmd_sys* sys, double cutoff, double margin) {
  if (!sys) return LJ_EINVAL;
  if (sys->broken) return LJ_EDEVICE;
  if (sys->n <= 0) return LJ_ESTATE;
  if (!(cutoff > 0.0) || !(margin >= 0.0)) return LJ_EINVAL;
  const ljmd_params old = sys->prm;
  sys->prm.cutoff = cutoff;
  sys->prm.margin = margin;
  int r = setup_geometry(sys, sys->L);
  if (r != LJ_OK) {
    sys->prm = old;
    setup_geometry(sys, sys->L);
    return r;
  }
  sys->forces_current = false;
  resolve_list_form(sys);
  TRY(rebuild(sys));
  return LJ_OK;
}

int ljmd_compute_forces(ljmd_sys* sys) {
  if (!sys) return LJ_EINVAL;
  if (sys->broken) return LJ_EDEVICE;
  if (sys->n <= 0) return LJ_ESTATE;
  if (!sys->have_list) {
    TRY(rebuild(sys));
  } else {
    // displacement since the list was built (shadow copies are current): rebuild if invalid
    IntegrateArgs a{0.0, 0.0, 0.0, 0, 1};
    CK(cudaMemsetAsync(sys->d_dmax, 0, 8, sys->st));
    integrate(sys, a);
    CKL();
    TRY(read_dmax(sys, &sys->last_dmax));
    bool expired = sys->last_dmax > sys->disp_limit;
    if (expired && (sys->valid_mode == LJ_VALID_DUTC_LDC || sys->valid_mode == LJ_VALID_HALF_MARGIN_LDC)) {
      bool ok = false;
      TRY(ldc_valid(sys, &ok));
      expired = !ok;
    }
    if (expired) TRY(rebuild(sys));
  }
  return run_force(sys, true);
}

int ljmd_step(ljmd_sys* sys, double dt, int64_t nsteps) {
  if (!sys || nsteps < 0 || !isfinite(dt)) return LJ_EINVAL;
  if (sys->broken) return LJ_EDEVICE;
  if (sys->n <= 0) return LJ_ESTATE;
  if (nsteps == 0) return LJ_OK;
  TRY(step_steps(sys, dt, nsteps));
  return check_status(sys);
}

}  // extern "C"

// The steps of ljmd_step without its final read of the device status word.
static int step_steps(ljmd_sys* sys, double dt, int64_t nsteps) {
  const int ee = sys->prm.energy_every;
  auto want_energy = [&](int64_t t) { return ee > 0 && (t % ee) == 0; };
  TRY(ensure_forces(sys, want_energy(sys->steps)));
  const double h = 0.5 * dt;
  cudaStream_t st = sys->st;
  // The margin/2 and DUTC rules are decided on the device (device_run); the rules with the large
  // displacement check need the host between steps.
  const bool on_device = sys->valid_mode == LJ_VALID_HALF_MARGIN || sys->valid_mode == LJ_VALID_DUTC;
  for (int64_t s = 0; s < nsteps;) {
    if (on_device) {
      int64_t advanced = 0;
      bool stopped = false;
      TRY(device_run(sys, dt, s == 0, nsteps - s, &advanced, &stopped));
      s += advanced;
      if (stopped) {  // the drift of the last step expired the list: rebuild, then its force
        TRY(rebuild(sys));
        TRY(run_force(sys, want_energy(sys->steps)));
      }
      continue;
    }
    const bool rec = sys->pe_step == sys->steps && want_energy(sys->steps);
    const int dutc = sys->valid_mode == LJ_VALID_DUTC || sys->valid_mode == LJ_VALID_DUTC_LDC;
    IntegrateArgs a{s == 0 ? 0.0 : h, h, dt, rec ? 1 : 0, 1, dutc};
    CK(cudaMemsetAsync(sys->d_dmax, 0, 8, st));
    const int nb = integrate(sys, a);
    CKL();
    if (rec) {
      energy_record(sys, nb, true);
      CKL();
    }
    sys->steps += 1;
    sys->forces_current = false;
    if (sys->cap_x) {
      launch_unwrapped(sys->x, sys->img, sys->id, sys->n, sys->g.offset, sys->L,
                       sys->cap_x + 3 * sys->n * (sys->steps - sys->cap_step0), st);
      sys->launches += 1;
    }
    TRY(read_dmax(sys, &sys->last_dmax));
    bool expired = false;
    TRY(list_expired(sys, dt, &expired));
    if (expired) TRY(rebuild(sys));
    TRY(run_force(sys, want_energy(sys->steps)));
    s += 1;
  }
  // final half-kick: v at the full step of the last state
  const bool rec = sys->pe_step == sys->steps && want_energy(sys->steps);
  IntegrateArgs a{h, 0.0, 0.0, rec ? 1 : 0, 0};
  const int nb = integrate(sys, a);
  CKL();
  if (rec) {
    energy_record(sys, nb, true);
    CKL();
  }
  return LJ_OK;
}

extern "C" {

int ljmd_energies(ljmd_sys* sys, double* pe, double* ke, double* virial) {
  if (!sys) return LJ_EINVAL;
  if (sys->broken) return LJ_EDEVICE;
  if (sys->n <= 0) return LJ_ESTATE;
  if (sys->energy_step != sys->steps) TRY(finalize_energies_now(sys));
  CK(cudaMemcpyAsync(sys->h_f64, sys->d_energies, 4 * sizeof(double), cudaMemcpyDeviceToHost, sys->st));
  CK(cudaStreamSynchronize(sys->st));
  if (pe) *pe = sys->h_f64[0];
  if (ke) *ke = sys->h_f64[1];
  if (virial) *virial = sys->h_f64[2];
  return check_status(sys);
}

int ljmd_set_energy_log(ljmd_sys* sys, double* device_log, int64_t capacity) {
  if (!sys || capacity < 0) return LJ_EINVAL;
  if (sys->broken) return LJ_EDEVICE;
  sys->log_ptr = device_log;
  sys->log_cap = device_log ? capacity : 0;
  if (cudaMemsetAsync(sys->d_log_count, 0, 8, sys->st) != cudaSuccess) return LJ_EDEVICE;
  return LJ_OK;
}

int ljmd_get_pairs(ljmd_sys* sys, int64_t* ij, int64_t cap, int64_t* npairs) {
  if (!sys || !npairs || cap < 0 || (cap > 0 && !ij)) return LJ_EINVAL;
  if (sys->broken) return LJ_EDEVICE;
  if (sys->n <= 0) return LJ_ESTATE;
  if (!sys->have_list) TRY(rebuild(sys));
  const int64_t N = sys->n;
  const uint64_t E = sys->list_entries;
  uint32_t* d_pairs = nullptr;
  TRY(dalloc_t(sys, &d_pairs, 2 * E + 2));
  if (cudaMemsetAsync(d_pairs, 0xff, sizeof(uint32_t) * (2 * E + 2), sys->st) != cudaSuccess) {
    cudaFree(d_pairs);
    sys->broken = true;
    return LJ_EDEVICE;
  }
  launch_list_decode(sys->cell_start, N, sys->ta, sys->rows, sys->ent, E, d_pairs, sys->d_status, sys->st);
  sys->launches += 1;
  std::vector<uint32_t> pr(2 * E);
  std::vector<int32_t> id(N);
  cudaError_t e1 = cudaGetLastError();
  if (e1 == cudaSuccess && E) e1 = cudaMemcpyAsync(pr.data(), d_pairs, sizeof(uint32_t) * 2 * E, cudaMemcpyDeviceToHost,
                                                   sys->st);
  if (e1 == cudaSuccess) e1 = cudaMemcpyAsync(id.data(), sys->id, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, sys->st);
  if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(sys->st);
  cudaFree(d_pairs);
  if (e1 != cudaSuccess) {
    sys->broken = true;
    return LJ_EDEVICE;
  }
  std::vector<std::pair<int64_t, int64_t>> pairs;
  pairs.reserve(!sys->list_half ? sys->list_actual / 2 : sys->list_actual);
  for (uint64_t k = 0; k < E; ++k) {
    if (pr[2 * k] == 0xffffffffu) continue;  // padding between tile segments
    if (pr[2 * k] >= (uint64_t)N || pr[2 * k + 1] >= (uint64_t)N) {
      fprintf(stderr, "ljmd_get_pairs: list entry %llu decodes to (%u, %u), N = %lld\n", (unsigned long long)k,
              pr[2 * k], pr[2 * k + 1], (long long)N);
      return LJ_EDEVICE;
    }
    const int64_t a = id[pr[2 * k]], b = id[pr[2 * k + 1]];
    if (!sys->list_half) {
      if (a < b) pairs.emplace_back(a, b);
    } else {
      pairs.emplace_back(std::min(a, b), std::max(a, b));
    }
  }
  std::sort(pairs.begin(), pairs.end());
  *npairs = (int64_t)pairs.size();
  const int64_t m = std::min<int64_t>(cap, (int64_t)pairs.size());
  for (int64_t k = 0; k < m; ++k) {
    ij[2 * k] = pairs[k].first;
    ij[2 * k + 1] = pairs[k].second;
  }
  return check_status(sys);
}

int ljmd_get_grid(ljmd_sys* sys, int64_t* grid_pointer, int64_t pointer_cap, int64_t* grid_list, int64_t list_cap,
                  int64_t* ncells) {
  if (!sys || !ncells || pointer_cap < 0 || list_cap < 0 || (pointer_cap > 0 && !grid_pointer) ||
      (list_cap > 0 && !grid_list))
    return LJ_EINVAL;
  if (sys->broken) return LJ_EDEVICE;
  if (sys->n <= 0 || !sys->have_list) return LJ_ESTATE;
  *ncells = sys->ncells;
  const int64_t np = std::min<int64_t>(pointer_cap, sys->ncells + 1);
  const int64_t nl = std::min<int64_t>(list_cap, sys->n);
  std::vector<uint32_t> ptr((size_t)std::max<int64_t>(np, 1));
  std::vector<int32_t> ids((size_t)std::max<int64_t>(nl, 1));
  if (np > 0) CK(cudaMemcpyAsync(ptr.data(), sys->cell_start, sizeof(uint32_t) * np, cudaMemcpyDeviceToHost, sys->st));
  if (nl > 0) CK(cudaMemcpyAsync(ids.data(), sys->id, sizeof(int32_t) * nl, cudaMemcpyDeviceToHost, sys->st));
  CK(cudaStreamSynchronize(sys->st));
  for (int64_t c = 0; c < np; ++c) grid_pointer[c] = (int64_t)ptr[(size_t)c];
  for (int64_t k = 0; k < nl; ++k) grid_list[k] = (int64_t)ids[(size_t)k];
  return check_status(sys);
}

int ljmd_get_stats(ljmd_sys* sys, ljmd_stats* out) {
  if (!sys || !out) return LJ_EINVAL;
  memset(out, 0, sizeof(*out));
  out->n = sys->n;
  out->steps = sys->steps;
  out->rebuilds = sys->rebuilds;
  out->list_entries = (int64_t)sys->list_actual;
  out->cells_per_side = sys->g.n;
  out->box = sys->L;
  out->mean_lifetime = sys->rebuilds > 0 ? (double)sys->steps / (double)sys->rebuilds : 0.0;
  out->max_displacement = sys->last_dmax;
  out->precision = sys->precision;
  out->kernel_launches = sys->launches;
  out->ldc_checks = sys->ldc_checks;
  out->ldc_kept = sys->ldc_kept;
  out->validity = sys->valid_mode;
  out->list_form = sys->list_half ? LJ_LIST_HALF : LJ_LIST_FULL;
  if (sys->broken) {
    out->status_word = -1;
    return LJ_EDEVICE;
  }
  int32_t w = 0;
  TRY(device_status(sys, &w));
  out->status_word = w;
  return LJ_OK;
}

int ljmd_set_tuning(ljmd_sys* sys, int32_t tile_cells, int32_t lanes, int32_t force_ctas_per_sm,
                    int32_t force_buffers) {
  if (!sys) return LJ_EINVAL;
  if (sys->broken) return LJ_EDEVICE;
  if (tile_cells < 0 || tile_cells > kMaxTileT || force_ctas_per_sm < 0 || force_ctas_per_sm > 4) return LJ_EINVAL;
  if (force_buffers < 0 || force_buffers > 2) return LJ_EINVAL;
  if (!(lanes == 0 || lanes == 1 || lanes == 2 || lanes == 4 || lanes == 8 || lanes == 16 || lanes == 32))
    return LJ_EINVAL;
  if (tile_cells != sys->tile_T) {
    sys->tile_T = tile_cells;
    sys->have_list = false;  // list indices depend on the tile shape
    sys->forces_current = false;
  }
  if (lanes) sys->prm.lanes = lanes;
  sys->force_per_sm = force_ctas_per_sm;
  if (force_buffers != sys->force_nbuf) {
    sys->force_nbuf = force_buffers;
    sys->have_list = false;  // the tile shape is re-checked against the larger shared-memory use
    sys->forces_current = false;
  }
  return LJ_OK;
}

int ljmd_set_profiling(ljmd_sys* sys, int32_t enable) {
  if (!sys) return LJ_EINVAL;
  if (sys->broken) return LJ_EDEVICE;
  resolve_events(sys);
  sys->profiling = enable != 0;
  for (int k = 0; k < 5; ++k) {
    sys->prof_ms[k] = 0.0;
    sys->prof_n[k] = 0;
  }
  return LJ_OK;
}

int ljmd_get_profile(ljmd_sys* sys, ljmd_profile* out) {
  if (!sys || !out) return LJ_EINVAL;
  if (sys->broken) return LJ_EDEVICE;
  resolve_events(sys);
  out->force_ms = sys->prof_ms[PH_FORCE];
  out->force_launches = sys->prof_n[PH_FORCE];
  out->integrate_ms = sys->prof_ms[PH_INTEGRATE];
  out->integrate_launches = sys->prof_n[PH_INTEGRATE];
  out->rebuild_ms = sys->prof_ms[PH_REBUILD];
  out->rebuilds = sys->prof_n[PH_REBUILD];
  out->energy_ms = sys->prof_ms[PH_ENERGY];
  out->energy_launches = sys->prof_n[PH_ENERGY];
  out->adjoint_ms = sys->prof_ms[PH_ADJOINT];
  out->adjoint_launches = sys->prof_n[PH_ADJOINT];
  return LJ_OK;
}


int ljmd_set_wait_budget(int64_t cycles) {
  if (cycles < 0) return LJ_EINVAL;
  return set_wait_budget((long long)cycles) == 0 ? LJ_OK : LJ_EDEVICE;
}

int ljmd_get_pairs_static(ljmd_sys* sys, int64_t* ij, int64_t cap, int64_t* npairs) {
  if (!sys || !npairs || cap < 0 || (cap > 0 && !ij)) return LJ_EINVAL;
  if (sys->broken) return LJ_EDEVICE;
  if (sys->n <= 0 || !sys->have_list) return LJ_ESTATE;
  const uint64_t E = sys->list_entries;
  if (E > (uint64_t)LJ_PAIRS_STATIC_MAX_ENTRIES) {
    fprintf(stderr, "ljmd_get_pairs_static: the list has %llu entries; the static scratch holds %d\n",
            (unsigned long long)E, LJ_PAIRS_STATIC_MAX_ENTRIES);
    return LJ_ERANGE;
  }
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev != sys->device) return LJ_EINVAL;
  unsigned long long *counter = nullptr, *keys = nullptr;
  TRY(pairs_static_scratch(dev, &counter, &keys));
  if (E == 0) {
    *npairs = 0;
    return check_status(sys);
  }
  uint32_t P = 2;
  while (P < E) P <<= 1;
  // The counter must start at zero; every key slot starts all-ones (tile padding is never written
  // by the decode, and the slots from E to P pad the sort).
  CK(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), sys->st));
  CK(cudaMemsetAsync(keys, 0xff, sizeof(unsigned long long) * P, sys->st));
  launch_list_decode(sys->cell_start, sys->n, sys->ta, sys->rows, sys->ent, E, (uint32_t*)keys, sys->d_status,
                     sys->st);
  CKL();
  launch_entries_to_keys(keys, E, sys->id, sys->n, !sys->list_half ? 1 : 0,
                         (unsigned int*)counter, sys->d_status, sys->st);
  CKL();
  sys->launches += 2 + launch_bitonic_sort(keys, P, sys->st);
  CKL();
  // the kept-pair count and the status word together; a raised status (an entry that decoded out
  // of range) returns before anything is written, as in ljmd_get_pairs
  CK(cudaMemcpyAsync(sys->h_u32, counter, sizeof(uint32_t), cudaMemcpyDeviceToHost, sys->st));
  CK(cudaMemcpyAsync(sys->h_i32, sys->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, sys->st));
  CK(cudaStreamSynchronize(sys->st));
  if (*sys->h_i32) return LJ_EDEVICE;
  const int64_t count = (int64_t)sys->h_u32[0];
  const int64_t m = std::min<int64_t>(cap, count);
  if (m > 0) {
    CK(cudaMemcpyAsync(ij, keys, sizeof(unsigned long long) * m, cudaMemcpyDeviceToHost, sys->st));
    CK(cudaStreamSynchronize(sys->st));
    // keys occupy ij[0, m); widen in place from the back (slot k is read before 2k, 2k+1 are written)
    for (int64_t k = m - 1; k >= 0; --k) {
      const uint64_t key = (uint64_t)ij[k];
      ij[2 * k] = (int64_t)(key >> 32);
      ij[2 * k + 1] = (int64_t)(key & 0xffffffffu);
    }
  }
  *npairs = count;
  return check_status(sys);
}


// ---- adjoint: Hessian-vector product and the reverse-time pass through velocity-Verlet --------
}  // extern "C"

static int ensure_adjoint(ljmd_sys* s) {
  if (s->adj_cap < s->n) {
    TRY(dalloc_t(s, &s->adj_w, s->n));
    TRY(dalloc_t(s, &s->adj_wf, s->n));
    TRY(dalloc_t(s, &s->adj_hw, s->n));
    TRY(dalloc_t(s, &s->adj_f, s->n));
    s->adj_cap = s->n;
  }
  if (!s->adj_ticket) {
    TRY(dalloc_t(s, &s->adj_ticket, 1));
    if (cudaMemsetAsync(s->adj_ticket, 0, sizeof(unsigned int), s->st) != cudaSuccess) return LJ_EDEVICE;
  }
  if (!s->part_adj) TRY(dalloc_t(s, &s->part_adj, 5 * (size_t)kMaxRedBlocks));
  if (!s->d_adj) TRY(dalloc_t(s, &s->d_adj, 8));
  return LJ_OK;
}

// One adjoint pass at the current positions with the vector w (device, id order; null = 0):
// hw = H w and f = F (device, id order; either may be null), q = [w.F, w.dF/dsigma, PE,
// dPE/dsigma, PE] (w.dF/deps = w.F / eps, dPE/deps = PE / eps).  With q non-null the sums are read
// to the host (synchronises); with q null they stay in the device scalars s->d_adj[0..4].
static int adjoint_pass(ljmd_sys* s, const double* w_id, double* hw_id, double* f_id, double* q,
                        bool f_sorted = false) {
  ljmd_sys* sys = s;
  if (!s->have_list) TRY(rebuild(s));
  TRY(ensure_adjoint(s));
  const int64_t N = s->n;
  cudaStream_t st = s->st;
  launch_to_sorted(w_id, s->id, N, s->adj_w, s->adj_wf, st);
  {
    PhaseTimer timer(s, PH_ADJOINT);
    launch_adjoint_tile(s->precision, force_pos(s), s->cell_start, N, s->g, s->ta, s->c, s->rows, s->tile_list,
                        s->ent, s->adj_w, s->adj_wf, s->adj_hw, (f_id || f_sorted) ? s->adj_f : nullptr, s->part_adj,
                        s->adj_ticket, s->d_adj, s->d_status, st);
  }
  s->launches += 2;
  if (hw_id) {
    launch_scatter_back_f64x4_to_f64x3(s->adj_hw, hw_id, s->id, N, st);
    s->launches += 1;
  }
  if (f_id) {
    launch_scatter_back_f64x4_to_f64x3(s->adj_f, f_id, s->id, N, st);
    s->launches += 1;
  }
  CKL();
  if (!q) return LJ_OK;
  CK(cudaMemcpyAsync(s->h_f64, s->d_adj, 5 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int k = 0; k < 5; ++k) q[k] = s->h_f64[k];
  return check_status(s);
}

template <class T>
struct DevBuf {  // device scratch owned by one call
  T* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  int alloc(size_t n) {
    if (cudaMalloc(&p, (n ? n : 1) * sizeof(T)) != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      return LJ_ENOMEM;
    }
    return LJ_OK;
  }
};

// Store positions given unwrapped in id order (device) without re-sorting the particles: the
// current order and image counts are kept, the force kernels' copies are rewritten, and the list
// stays if no particle moved more than margin/2 from where it was built (else it is rebuilt).
// Velocities are left as they are.  Synchronises once (the displacement maximum).
// known_valid: the state was reached by a step that the validity rule accepted for the current list
// (no rebuild since), so its displacement need not be read back.
static int load_keeping_list(ljmd_sys* s, const double* u, bool known_valid = false) {
  ljmd_sys* sys = s;
  if (!s->have_list) {  // nothing to keep: the general path
    return ljmd_set_state(s, s->n, s->L, u, nullptr, 1);
  }
  launch_load_unwrapped(u, s->img, s->id, s->n, s->g.offset, s->L, s->x, s->st);
  s->launches += 1;
  CKL();
  if (!known_valid) CK(cudaMemsetAsync(s->d_dmax, 0, 8, s->st));  // (a run clears it before its use)
  IntegrateArgs a{0.0, 0.0, 0.0, 0, 1};  // no kick, no drift: copies and displacement only
  integrate(s, a);
  CKL();
  s->forces_current = false;
  s->pe_step = -1;
  s->energy_step = -1;
  if (known_valid) return LJ_OK;
  TRY(read_dmax(s, &s->last_dmax));
  if (s->last_dmax > s->disp_limit) TRY(rebuild(s));
  return LJ_OK;
}

extern "C" {

int ljmd_hvp(ljmd_sys* sys, const double* w, double* hw, double* dtheta, int32_t on_device) {
  if (!sys || !w || !hw) return LJ_EINVAL;
  if (sys->broken) return LJ_EDEVICE;
  if (sys->n <= 0) return LJ_ESTATE;
  TRY(adjoint_list_form(sys));
  const int64_t N = sys->n;
  const size_t bytes = sizeof(double) * 3 * (size_t)N;
  DevBuf<double> wd, hd;
  const double* w_dev = w;
  double* hw_dev = hw;
  if (!on_device) {
    TRY(wd.alloc(3 * (size_t)N));
    TRY(hd.alloc(3 * (size_t)N));
    CK(cudaMemcpyAsync(wd.p, w, bytes, cudaMemcpyHostToDevice, sys->st));
    w_dev = wd.p;
    hw_dev = hd.p;
  }
  double q[5];
  TRY(adjoint_pass(sys, w_dev, hw_dev, nullptr, q));
  if (!on_device) {
    CK(cudaMemcpyAsync(hw, hd.p, bytes, cudaMemcpyDeviceToHost, sys->st));
    CK(cudaStreamSynchronize(sys->st));
  }
  if (dtheta) {
    const double eps = sys->prm.eps;
    dtheta[0] = q[0] / eps;
    dtheta[1] = q[1];
    dtheta[2] = q[4] / eps;
    dtheta[3] = q[3];
  }
  return LJ_OK;
}

int ljmd_traj_loss_grad(ljmd_sys* sys, int64_t n, double box, const double* x0, const double* v0, double dt,
                        int64_t nsteps, int64_t n_pe, int64_t ckpt_every, double* loss, double* gx0, double* gv0,
                        double* gtheta, int32_t on_device) {
  if (!sys || n <= 0 || !x0 || !v0 || !loss || nsteps < 1 || n_pe < 0 || n_pe > nsteps || ckpt_every < 1 ||
      !isfinite(dt))
    return LJ_EINVAL;
  if (sys->broken) return LJ_EDEVICE;
  TRY(adjoint_list_form(sys));
  const size_t n3 = 3 * (size_t)n;
  const size_t bytes = sizeof(double) * n3;
  const int64_t nseg = (nsteps + ckpt_every - 1) / ckpt_every;
  cudaStream_t st = sys->st;
  DevBuf<double> ck_x, ck_v, seg_x, x0u, xNu, lx, lv, b, f, part, elog;
  DevBuf<int64_t> ecount;
  const int64_t elog_cap = nsteps + 2 * nseg + 4;
  TRY(ck_x.alloc(n3 * (size_t)nseg));
  TRY(ck_v.alloc(n3 * (size_t)nseg));
  TRY(seg_x.alloc(n3 * (size_t)ckpt_every));
  TRY(x0u.alloc(n3));
  TRY(xNu.alloc(n3));
  TRY(lx.alloc(n3));
  TRY(lv.alloc(n3));
  TRY(b.alloc(n3));
  TRY(f.alloc(n3));
  TRY(part.alloc(kMaxRedBlocks + 8));
  TRY(elog.alloc(4 * (size_t)elog_cap));
  TRY(ecount.alloc(1));
  // the initial state on the device
  if (on_device) {
    CK(cudaMemcpyAsync(x0u.p, x0, bytes, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ck_v.p, v0, bytes, cudaMemcpyDeviceToDevice, st));
  } else {
    CK(cudaMemcpyAsync(x0u.p, x0, bytes, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ck_v.p, v0, bytes, cudaMemcpyHostToDevice, st));
  }
  CK(cudaMemcpyAsync(ck_x.p, x0u.p, bytes, cudaMemcpyDeviceToDevice, st));
  auto capture = [&](double* xu, double* vv) -> int {
    launch_unwrapped(sys->x, sys->img, sys->id, sys->n, sys->g.offset, sys->L, xu, st);
    if (vv) launch_scatter_back_f64x3(sys->v, vv, sys->id, sys->n, 0.0, st);
    sys->launches += vv ? 2 : 1;
    CK(cudaGetLastError());
    return LJ_OK;
  };
  const double h = 0.5 * dt, wpe = n_pe > 0 ? 1.0 / ((double)n_pe * (double)n) : 0.0;
  // the caller's energy settings are replaced while this call runs: every state's PE goes to an
  // internal log (one device-decided run per checkpoint segment, no host round trip per step)
  const int saved_ee = sys->prm.energy_every;
  double* const saved_log = sys->log_ptr;
  const int64_t saved_cap = sys->log_cap;
  int64_t* const saved_count = sys->d_log_count;
  auto restore = [&]() {
    sys->prm.energy_every = saved_ee;
    sys->log_ptr = saved_log;
    sys->log_cap = saved_cap;
    sys->d_log_count = saved_count;
  };
  auto run_or_restore = [&](int r) {
    if (r != LJ_OK) restore();
    return r;
  };
  // ---- forward: checkpoints every ckpt_every steps, PE of the last n_pe states from the log
  TRY(ljmd_set_state(sys, n, box, ck_x.p, ck_v.p, 1));
  sys->prm.energy_every = n_pe > 0 ? 1 : 0;
  sys->log_ptr = elog.p;
  sys->log_cap = elog_cap;
  sys->d_log_count = ecount.p;
  if (cudaMemsetAsync(ecount.p, 0, sizeof(int64_t), st) != cudaSuccess) {
    restore();
    sys->broken = true;
    return LJ_EDEVICE;
  }
  for (int64_t seg = 0; seg < nseg; ++seg) {
    const int64_t t0 = seg * ckpt_every, t1 = std::min<int64_t>(t0 + ckpt_every, nsteps);
    TRY(run_or_restore(step_steps(sys, dt, t1 - t0)));
    if (t1 < nsteps) TRY(run_or_restore(capture(ck_x.p + n3 * (size_t)(seg + 1), ck_v.p + n3 * (size_t)(seg + 1))));
  }
  int64_t nrec = 0;
  std::vector<double> recs;
  {
    cudaError_t e = cudaMemcpyAsync(&nrec, ecount.p, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    nrec = std::min<int64_t>(nrec, elog_cap);
    recs.resize(4 * (size_t)std::max<int64_t>(nrec, 1));
    if (e == cudaSuccess && nrec > 0)
      e = cudaMemcpyAsync(recs.data(), elog.p, sizeof(double) * 4 * nrec, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    restore();
    if (e != cudaSuccess) {
      sys->broken = true;
      return LJ_EDEVICE;
    }
  }
  // PE of the states nsteps - n_pe + 1 .. nsteps (a state is recorded twice at a segment boundary)
  double acc_pe = 0.0;
  if (n_pe > 0) {
    std::vector<char> seen((size_t)nsteps + 1, 0);
    for (int64_t k = 0; k < nrec; ++k) {
      const int64_t t = (int64_t)recs[4 * k];
      if (t > nsteps - n_pe && t <= nsteps && !seen[(size_t)t]) {
        seen[(size_t)t] = 1;
        acc_pe += recs[4 * k + 1];
      }
    }
    for (int64_t t = nsteps - n_pe + 1; t <= nsteps; ++t)
      if (!seen[(size_t)t]) return LJ_EDEVICE;  // a state's energy record is missing
  }
  TRY(capture(xNu.p, nullptr));
  const int nb = launch_sqdiff(xNu.p, x0u.p, (int64_t)n3, part.p, st);
  launch_final_reduce(part.p, nb, 1, part.p + kMaxRedBlocks, st);
  CKL();
  CK(cudaMemcpyAsync(sys->h_f64, part.p + kMaxRedBlocks, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const double msd = sys->h_f64[0] / (double)n;
  *loss = acc_pe * wpe + msd;
  if (!gx0 && !gv0 && !gtheta) return check_status(sys);

  // ---- reverse: lx = dloss/dx_n, lv = 0; then state by state back to t = 0.  The parameter
  // gradient is summed on the device (one read at the end).
  const double eps = sys->prm.eps;
  DevBuf<double> gthd;
  TRY(gthd.alloc(2));
  CK(cudaMemsetAsync(gthd.p, 0, 2 * sizeof(double), st));
  launch_scaled_diff(lx.p, 2.0 / (double)n, xNu.p, x0u.p, (int64_t)n3, st);
  CK(cudaMemsetAsync(lv.p, 0, bytes, st));
  if (n_pe > 0) {
    TRY(adjoint_pass(sys, nullptr, nullptr, f.p, nullptr));  // at x_n: F and dPE
    launch_axpy(lx.p, -wpe, f.p, (int64_t)n3, st);
    launch_accum_q(sys->d_adj, 0.0, 0.0, wpe, wpe / eps, gthd.p, st);
    sys->launches += 2;
  }
  for (int64_t seg = nseg - 1; seg >= 0; --seg) {
    const int64_t t0 = seg * ckpt_every, t1 = std::min<int64_t>(t0 + ckpt_every, nsteps);
    // recompute the segment's states t0 .. t1 - 1 from its checkpoint
    TRY(ljmd_set_state(sys, n, box, ck_x.p + n3 * (size_t)seg, ck_v.p + n3 * (size_t)seg, 1));
    CK(cudaMemcpyAsync(seg_x.p, ck_x.p + n3 * (size_t)seg, bytes, cudaMemcpyDeviceToDevice, st));
    // one run over the segment (the forward pass's call structure, so the same states), the
    // state after every step captured on the device
    sys->prm.energy_every = 0;
    if (t1 - t0 > 1) {
      sys->cap_x = seg_x.p;
      sys->cap_step0 = 0;  // the state counter restarts at the checkpoint
      const int r = step_steps(sys, dt, t1 - t0 - 1);
      sys->cap_x = nullptr;
      TRY(run_or_restore(r));
    }
    sys->prm.energy_every = saved_ee;
    // states from the last construction on were accepted by the validity rule for the current list
    const int64_t valid_from = sys->last_build_step;
    const int64_t builds = sys->rebuilds;
    for (int64_t t = t1 - 1; t >= t0; --t) {
      launch_axpy(lv.p, dt, lx.p, (int64_t)n3, st);  // x_{t+1} = x_t + dt v'
      // state t in the particle order of the recomputation: its list is kept while it is valid
      TRY(load_keeping_list(sys, seg_x.p + n3 * (size_t)(t - t0), t - t0 >= valid_from && sys->rebuilds == builds));
      const double c = t == 0 ? h : dt;  // both half-kicks touching state t (one at t = 0)
      const bool in_pe = t > nsteps - n_pe;
      // H lv (and F where the PE term needs it) in the sorted order, then lx -= c H lv + wpe F
      TRY(adjoint_pass(sys, lv.p, nullptr, nullptr, nullptr, in_pe));
      launch_adjoint_update(sys->adj_hw, in_pe ? sys->adj_f : nullptr, sys->id, sys->n, c, in_pe ? wpe : 0.0, lx.p,
                            st);
      launch_accum_q(sys->d_adj, c / eps, c, in_pe ? wpe : 0.0, in_pe ? wpe / eps : 0.0, gthd.p, st);
      if (t == 0) {
        // MSD term at t = 0: -2 (x_n - x_0) / N
        launch_scaled_diff(b.p, -2.0 / (double)n, xNu.p, x0u.p, (int64_t)n3, st);
        launch_axpy(lx.p, 1.0, b.p, (int64_t)n3, st);
      }
      sys->launches += 3 + (t == 0 ? 2 : 0);
      CKL();
    }
  }
  if (gx0) CK(cudaMemcpyAsync(gx0, lx.p, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  if (gv0) CK(cudaMemcpyAsync(gv0, lv.p, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(sys->h_f64, gthd.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (gtheta) {
    gtheta[0] = sys->h_f64[0];
    gtheta[1] = sys->h_f64[1];
  }
  return check_status(sys);
}


int ljmd_set_validity(ljmd_sys* sys, int32_t mode, int32_t max_ld) {
  if (!sys) return LJ_EINVAL;
  if (sys->broken) return LJ_EDEVICE;
  if (mode < LJ_VALID_HALF_MARGIN || mode > LJ_VALID_HALF_MARGIN_LDC || max_ld < 0) return LJ_EINVAL;
  if (max_ld > 0 && max_ld != sys->max_ld) {
    if (sys->ldc_list) cudaFree(sys->ldc_list);
    sys->ldc_list = nullptr;
    sys->max_ld = max_ld;
  }
  if (mode != sys->valid_mode) {
    sys->valid_mode = mode;
    sys->have_list = false;  // the next construction records what the new rule needs
    sys->forces_current = false;
  }
  return LJ_OK;
}


}  // extern "C"
