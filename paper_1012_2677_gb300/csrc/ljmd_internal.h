// Internal declarations shared by the CUDA translation units of libljmd.
// Nothing here is part of the C ABI (include/ljmd.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ljmd.h"

namespace ljmd {

// 32-byte aligned four-double vector (one 32-byte access per particle).
typedef double4_32a dvec4;

// Kernels that produce per-block partial sums run on at most this many blocks
// (grid-stride loops), so partial buffers have a fixed size and the final
// reduction has a fixed order (results do not depend on timing).
constexpr int kMaxRedBlocks = 1216;  // 152 SMs x 8
constexpr int kRedThreads = 256;

// Box geometry.  Positions are stored as x_state = offset + x with
// offset = 2^p >= L + margin (and >= 4), so every stored coordinate lies in
// [offset/2, 2 offset) and shares one binade-pair: differences of stored
// coordinates are exact in FP64, and their FP32 "hi" parts (the top 24
// significand bits) are all multiples of 2^(p-24), which makes the FP32
// difference of two hi parts exact as well.
struct Geom {
  double L;        // box side
  double half_L;   // L / 2 (exact)
  double offset;   // 2^p
  double inv_h;    // cells per side / L
  int32_t n;       // cells per side
  int32_t p;       // log2(offset)
  float L_hi;      // L truncated to a multiple of 2^(p-23) (exact FP32)
  float L_lo;      // L - L_hi rounded to FP32
  float inv_L;     // 1 / L in FP32 (picks the periodic image)
  double inv_L64;  // 1 / L in FP64
  // Fixed-point positions of the mixed form's pair arithmetic: X = round(x_state / u) mod 2^32 with
  // u = 2^-qk.  Two such coordinates differ by an exact 32-bit integer as long as the true
  // difference is below 2^31 u, which qk guarantees for every difference the kernels take
  // (staged neighbour cells, list partners, displacements since the build, the whole box).
  int32_t qk;      // u = 2^-qk
  uint32_t Lq;     // round(L / u) mod 2^32: the periodic image shift in units of u
  float qu;        // u (a power of two: scaling by it is exact)
  float q_inv_L;   // u / L in FP32 (picks the periodic image of a whole-box difference)
};

// Potential constants (Eq. 2) in the forms the kernels use.
struct LJConst {
  double eps, sigma, rc2, c2, c0, sig2;  // FP64 form
  float f24, f48, f8c2;                  // force: f = ri2 s3i (f24 - f48 s3i) + f8c2
  float sig2f, rc2f, e4, c2f, c0f;       // energy: 4 eps (s3i (s3i - 1) + c2 s + c0)
  // The same constants for differences in units of u (fixed-point positions): with d_u = d / u and
  // r2_u = r^2 / u^2, f_u d_u = f d when f24q = f24 / u, f48q = f48 / u, f8c2q = f8c2 u, and
  // sig2q = sig2 / u^2, rc2q = rc2 / u^2, c2q = c2 u^2.  u is a power of two, so these are the
  // FP32 constants above with their exponents shifted (no extra rounding); the virial comes out
  // in units of 1/u and is multiplied by u (exactly) when it is summed.
  float f24q, f48q, f8c2q, sig2q, rc2q, c2q;
  // the adjoint kernel's constants: 1 / sigma and c2 / sigma^2, FP64 and FP32
  double inv_sigma, c2s;
  float inv_sigmaf, c2sf;
};

struct ListBand {
  double rs2;      // r_s^2 in FP64 (exact test)
  float lo, hi;    // FP32 band: r2f < lo accept, r2f >= hi reject, else exact FP64 test
};

// ---- reductions / status -------------------------------------------------------
void launch_final_reduce(const double* partials, int nblocks, int nq, double* out, cudaStream_t s);
// skip (optional): a device flag; set, the launch does nothing (a device-decided run stopped).
void launch_energy_finalize(const double* pe_vir_part, int nb_force, const double* ke_part, int nb_int,
                            double pe_scale, double* energies, double* log, int64_t log_cap, int64_t* log_count,
                            double step, cudaStream_t s, const int* skip = nullptr);

// ---- init ---------------------------------------------------------------------------
void launch_fcc(double* x, int64_t M, double a, double offset, cudaStream_t s);
void launch_gaussian(double* v, int64_t N, uint64_t seed, cudaStream_t s);
void launch_sums3(const double* v, int64_t N, double* partials, int nb, cudaStream_t s);
void launch_sumsq_centered(const double* v, int64_t N, const double* sums, double* partials, int nb, cudaStream_t s);
void launch_center_scale(double* v, int64_t N, const double* sums, const double* sumsq, double T, cudaStream_t s);
int red_blocks(int64_t n);

// ---- grid ---------------------------------------------------------------------------
void launch_wrap_label(double* x, int32_t* img, int64_t N, Geom g, uint32_t* cell_of, uint32_t* cell_count,
                       int32_t* status, cudaStream_t s);
// exclusive scan of n uint32 values into out[0..n] (out[n] = total); tmp >= scan_tmp_words(n)
size_t scan_tmp_words(int64_t n);
// returns the number of kernels launched
int launch_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, cudaStream_t s,
    const int* pred = nullptr);
void launch_scatter(const uint32_t* cell_of, const uint32_t* cell_start, uint32_t* cell_fill, uint32_t* perm,
                    int64_t N, cudaStream_t s,
    const int* pred = nullptr);
// Cell by cell, the entries of perm_in ordered by id, written to perm_out.
void launch_cell_rank(const uint32_t* cell_start, int64_t ncells, const uint32_t* perm_in, const int32_t* id,
                      uint32_t* perm_out, cudaStream_t s, const int* pred = nullptr);
void launch_gather_state(const uint32_t* perm, int64_t N, const double* x, double* x2, const double* v, double* v2,
                         const int32_t* id, int32_t* id2, const int32_t* img, int32_t* img2, const void* f, void* f2,
                         int fbytes, cudaStream_t s, const int* pred);
void launch_scatter_back_f64x3(const double* in, double* out_idorder, const int32_t* id, int64_t N,
                               double sub, cudaStream_t s);
void launch_scatter_back_f32x4_to_f64x3(const float4* in, double* out, const int32_t* id, int64_t N,
                                        cudaStream_t s);
void launch_scatter_back_f64x4_to_f64x3(const dvec4* in, double* out, const int32_t* id, int64_t N,
                                        cudaStream_t s);
void launch_scatter_back_i32x3(const int32_t* in, int32_t* out, const int32_t* id, int64_t N, cudaStream_t s);
void launch_iota_i32(int32_t* id, int64_t N, cudaStream_t s);
void launch_load_state(const double* x_in, const double* v_in, double* x, double* v, int32_t* id, int32_t* img,
                       int64_t N, double offset, double L, cudaStream_t s);

// ---- shadow positions ---------------------------------------------------------------
// hi: the FP32 hi parts of x_state (the list kernels' filter, both forms); mixed: the fixed-point
// records xq (X, Y, Z at u = 2^-qk, w = sorted index); fp64: the dvec4 copy.  ref (optional)
// receives xq (mixed) or the dvec4 (fp64) as the displacement reference.
void launch_shadow_all(const double* x, int64_t N, int mixed, int qk, float4* hi, uint4* xq, dvec4* pos64, void* ref,
                       cudaStream_t s, const int* pred = nullptr);

// ---- staged cell-column tiles: list and force ---------------------------------------------
constexpr int kMaxTileT = 14;  // cells per tile along z, at most
struct TileArgs {
  int32_t n;           // cells per side
  int32_t T;           // cells per tile along z (1 <= T <= n - 2); tile path needs n >= 3
  int32_t ntz;         // tiles per column, ceil(n / T)
  int32_t whole;       // 1: the whole box is one tile (n < 3), periodic image chosen per pair
  int64_t ntiles;
  int32_t max_staged;  // staged particles per tile, at most (<= 65535: entries are 16-bit)
  int32_t max_own;     // own particles per tile, at most
  int32_t max_chunks;  // 32-candidate chunks per own particle, at most
  int32_t max_list;    // list entries per tile (padded to 8), at most (known after construction)
  int32_t list_cap;    // entries of a tile's segment the force kernel stages; longer ones stay in HBM
};
// One replica of a batch: its box (offset and p are the batch's), grid, tiles and particles.
// Global tiles, cells and particles are the replicas' ranges concatenated in replica order.
struct ReplicaGeo {
  Geom g;
  int32_t n, T, ntz, pad;  // cells per side, cells per tile along z, tiles per column
  int64_t tile_base;       // first global tile
  int64_t cell_base;       // first global cell
  int64_t base, count;     // first global particle, particles
};
size_t list_smem_bytes(const TileArgs& ta, int precision);
size_t force_smem_bytes(const TileArgs& ta, int precision, int nbuf, int half);
void launch_max_count(const uint32_t* cnt, int64_t n, unsigned int* out, cudaStream_t s);
void launch_tile_sizes(const uint32_t* cs, TileArgs ta, unsigned int* out, cudaStream_t s);
// counter[0] += padded tile segments (reservations), counter[1] += actual entries
void launch_list_tile(int precision, int half, const void* pos, const float4* hi, const double* x, const uint32_t* cs,
                      int64_t N, Geom g, TileArgs ta, ListBand band, uint2* rows, uint2* tile_list, uint16_t* ent,
                      uint64_t cap, unsigned long long* counter, unsigned int* max_list, int32_t* status,
                      cudaStream_t s);
// pos: the fixed-point records (mixed) or the dvec4 copies (FP64).  Returns the number of blocks
// (energy partials written to part[2 b], part[2 b + 1]).
int launch_force_tile(int precision, int half, int lanes, int energy, const void* pos, const uint32_t* cs, int64_t N,
                      Geom g, TileArgs ta, LJConst c, const uint2* rows, const uint2* tile_list, const uint16_t* ent,
                      void* f, double* part, int32_t* status, int per_sm, int nbuf, cudaStream_t s,
                      const int* skip = nullptr);
size_t adjoint_smem_bytes(const TileArgs& ta, int precision);
// Adjoint pass (HVP, forces, parameter derivatives) over the list; w, hw, fo are dvec4 [N] in sorted
// order (fo may be null), wf the FP32 copy of w (read by the mixed form).  Writes 5 partials per
// block [w.dF/deps, w.dF/dsigma, dPE/deps, dPE/dsigma, PE]; the last block to finish (ticket: zero
// between launches) writes their sums, in block order, to sums[0..4].  Returns the number of blocks.
int launch_adjoint_tile(int precision, const void* pos, const uint32_t* cs, int64_t N, Geom g, TileArgs ta, LJConst c,
                        const uint2* rows, const uint2* tile_list, const uint16_t* ent, const void* w,
                        const float4* wf, void* hw, void* fo, double* part, unsigned int* ticket, double* sums,
                        int32_t* status, cudaStream_t s);
void launch_list_decode(const uint32_t* cs, int64_t N, TileArgs ta, const uint2* rows, const uint16_t* ent,
                        uint64_t E, uint32_t* out, int32_t* status, cudaStream_t s);

// ---- integrator ---------------------------------------------------------------------
struct IntegrateArgs {
  double kpre;     // kick that brings v to the full step before the kinetic energy is taken
  double kpost;    // kick after it (the first half-kick of the next step)
  double dt;       // drift length (0 = no drift)
  int ke;          // accumulate the kinetic energy of the full-step velocity
  int shadow;      // rewrite the force kernel's position copy after the drift
  int speed;       // also reduce the largest drift speed (DUTC rules)
  int qk;          // mixed form: the fixed-point records are at u = 2^-qk
};
// Work done by the integrator's last CTA (an atomic ticket counts the CTAs that finished), in place
// of separate launches: the energy record of the step (force partials pv of the state before the
// drift, the KE partials of this launch) and the list-validity check of a device-decided run.
struct StepCtl;
struct StepFinish {
  unsigned int* ticket;  // zero between launches; nullptr: nothing to finish
  int rec;               // the energy record (as launch_energy_finalize)
  const double* pv;
  int nbf;
  double pe_scale;
  double* energies;
  double* log;
  int64_t cap;
  int64_t* count;
  double step;
  int check;  // the validity check: the run stops at step s if the list expired
  StepCtl* ctl;
  int s;
  double disp_limit;
  int dutc;
  double two_dt;
};
// Returns the number of blocks used for KE partials.  With a.shadow, dmax_bits[0] and [1] receive
// (atomic max) the float bits of the largest squared displacement since the list build and of the
// largest squared drift speed.
// pos: the fixed-point records (mixed) or the dvec4 copies (FP64), rewritten when a.shadow is set.
int launch_integrate(int precision, double* x, double* v, const void* f, void* pos, const void* ref, int64_t N,
                     IntegrateArgs a, double* ke_part, uint32_t* dmax_bits, int32_t* status, StepFinish fin, cudaStream_t s,
                     const int* skip = nullptr);
// Device-side list-validity decision after the drift of step s of a device-decided run (taken by the
// integrator's last CTA, StepFinish.check): unless ctl->stop is already set, reads the maxima of the
// step (squared displacement since the build and squared drift speed, float bits in dmax_bits[0],
// [1]), keeps them in ctl->last, clears dmax_bits for the next step and, if the list expired
// (margin/2 rule: the displacement above disp_limit; DUTC: the buffer, reduced by 2 v_max |dt|, at
// or below zero), sets ctl->stop and ctl->stop_at = s.  Every later kernel of the run is launched
// with &ctl->stop as its skip flag.
struct StepCtl {
  int stop;         // set: the run stopped (the list must be rebuilt before the next force)
  int stop_at;      // the step of the run whose drift expired the list
  float last[2];    // squared largest displacement and drift speed of the last checked step
  double dutc;      // DUTC buffer length
};
// ---- pair export through a static device scratch array (no allocation) ----------------
// Address of this device's scratch (resolved once per device): the kept-pair counter word and
// LJ_PAIRS_STATIC_MAX_ENTRIES 64-bit key slots.
int pairs_static_scratch(int device, unsigned long long** counter_word, unsigned long long** keys);
void launch_entries_to_keys(unsigned long long* keys, uint64_t E, const int32_t* id, int64_t N, int full,
                            unsigned int* counter, int32_t* status, cudaStream_t s);
// Ascending bitonic sort of P = 2^m keys in place; returns the number of kernel launches.
int launch_bitonic_sort(unsigned long long* keys, uint32_t P, cudaStream_t s);

// ---- adjoint pass helpers (kernels_adjoint.cu) ----------------------------------------
void launch_to_sorted(const double* w_id, const int32_t* id, int64_t N, dvec4* out, float4* out32, cudaStream_t s);
void launch_unwrapped(const double* x, const int32_t* img, const int32_t* id, int64_t N, double offset, double L,
                      double* out, cudaStream_t s, const StepCtl* ctl = nullptr, int k_step = 0);
// x (sorted order, SoA) = offset + u (unwrapped, id order) - img L with the current order and images
void launch_load_unwrapped(const double* u, const int32_t* img, const int32_t* id, int64_t N, double offset, double L,
                           double* x, cudaStream_t s);
void launch_axpy(double* y, double a, const double* x, int64_t n, cudaStream_t s);
// lx[3 id[s] + k] -= c hw[s].k + a f[s].k over the sorted order (f null: a ignored).
void launch_adjoint_update(const dvec4* hw, const dvec4* f, const int32_t* id, int64_t N, double c, double a,
                           double* lx, cudaStream_t s);
// gth[0] += a0 q[0] + a4 q[4], gth[1] += a1 q[1] + a3 q[3] (device scalars)
void launch_accum_q(const double* q, double a0, double a1, double a3, double a4, double* gth, cudaStream_t s);
void launch_scaled_diff(double* y, double a, const double* u, const double* w, int64_t n, cudaStream_t s);
int launch_sqdiff(const double* u, const double* w, int64_t n, double* part, cudaStream_t s);

// ---- batched replicas (kernels_tile.cu, kernels_batch.cu) ----------------------------------
size_t batch_list_smem_bytes(const TileArgs& caps);
size_t batch_force_smem_bytes(const TileArgs& caps);
void launch_tile_sizes_batch(const uint32_t* cs, TileArgs caps, const ReplicaGeo* reps, int R,
                             const int32_t* tile_rep, unsigned int* out, cudaStream_t s);
void launch_list_batch(const float4* hi, const double* x, const uint32_t* cs, int64_t N, Geom g, TileArgs caps,
                       ListBand band, uint2* rows, uint2* tile_list, uint16_t* ent, uint64_t cap,
                       unsigned long long* counter, unsigned int* max_list, int32_t* status, const ReplicaGeo* reps,
                       int R, const int32_t* tile_rep, const int* pred, cudaStream_t s);
int launch_force_batch(int lanes, int energy, const uint4* xq, const uint32_t* cs, int64_t N,
                       TileArgs caps, LJConst c, const uint2* rows, const uint2* tile_list, const uint16_t* ent,
                       float4* f, double* e_rep, int32_t* status, const ReplicaGeo* reps, int R,
                       const int32_t* tile_rep, cudaStream_t s);
void launch_wrap_label_batch(double* x, int32_t* img, int64_t N, const int32_t* rep_of, const ReplicaGeo* reps,
                             double offset, uint32_t* cell_of, uint32_t* cell_count, int32_t* status,
                             const int* pred, cudaStream_t s);
void launch_rebuild_flag(const uint32_t* dmax_bits, float limit2, int* flag, long long* rebuilds, cudaStream_t s);
void launch_copy_words(const void* in, void* out, int64_t bytes, const int* pred, cudaStream_t s);
void launch_zero_words(void* out, int64_t bytes, const int* pred, cudaStream_t s);
void launch_replica_ke(const double* v, int64_t N, const ReplicaGeo* reps, int R, double* ke_rep, cudaStream_t s);
void launch_load_batch(const double* xin, const double* vin, double* x, double* v, int32_t* id, int32_t* img,
                       int64_t N, const int32_t* rep_of, const ReplicaGeo* reps, double offset, cudaStream_t s);

// ---- list validity (kernels_tile.cu) --------------------------------------------------------
// Budget of the bounded device waits of the tile kernels (0: default); 0 on success.
int set_wait_budget(long long cycles);
void launch_ldc_collect(const double* x, const double* xref, int64_t N, double th2, int32_t* list, unsigned int cap,
                        unsigned int* count, cudaStream_t s);
void launch_ldc_pairs(const double* x, const double* xref, int64_t N, Geom g, const int32_t* list, int m, double rs2,
                      double rc2, int* flag, cudaStream_t s);

}  // namespace ljmd
