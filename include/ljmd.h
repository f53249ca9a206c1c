/*
 * ljmd.h -- C ABI of the GB300 Lennard-Jones molecular-dynamics library.
 *
 * The method is the one of Watanabe, Suzuki and Ito, "Efficient
 * Implementations of Molecular Dynamics Simulations for Lennard-Jones
 * Systems": the truncated LJ pair force (Sec. 2.1, Eq. 2) summed over a
 * bookkeeping (Verlet) pair list with a search length r_s = r_c + margin
 * (Sec. 2.3), built from a cell grid whose counting sort also reorders the
 * particles for locality (Sec. 2.2, Sec. 3.3), stored as a sorted list
 * (Sec. 2.4, KeyPointer/SortedList), and driven by a second-order symplectic
 * (velocity-Verlet) integrator (Sec. 4.5).
 *
 * Conventions for every call:
 *   - Reduced units (sigma, eps of the potential; m = 1, kB = 1).
 *   - A periodic cubic box of side L in [0, L)^3.
 *   - Host arrays are caller-owned, float64, particle-major: x[3*i + k].
 *     Device arrays (on_device = 1) have the same layout and must live on the
 *     device the handle was created on.  The library never frees caller memory.
 *   - Particle order in and out of the library is the caller's id order; the
 *     library keeps particles sorted by cell internally.
 *   - Every call is asynchronous on the stream given to ljmd_create except
 *     where it says it synchronises.
 *   - Return value: LJ_OK (0) or a negative LJ_E* code; ljmd_strerror()
 *     names it.  After LJ_EDEVICE the handle should be destroyed.
 *   - The handle owns all device memory it allocates and is not thread-safe.
 */
#ifndef LJMD_H
#define LJMD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define LJ_OK 0
#define LJ_EINVAL (-1)   /* bad argument (N <= 0, cutoff <= 0, margin < 0, L < 2 (r_s + margin), NULL) */
#define LJ_ENOMEM (-2)   /* device or host allocation failed */
#define LJ_EDEVICE (-3)  /* CUDA error, or the device status word was raised (see LJ_ST_*) */
#define LJ_ESTATE (-4)   /* call out of order (no particles yet) */
#define LJ_ERANGE (-5)   /* size beyond a library limit (e.g. more than 2^32 - 1 list entries) */

/* ---- device status word bits (ljmd_stats.status_word) ---- */
#define LJ_ST_NONFINITE 1   /* a position, velocity or force became NaN/Inf */
#define LJ_ST_LIST_OVERFLOW 2 /* a list fill exceeded its counted size (internal consistency check) */
#define LJ_ST_TIMEOUT 4     /* a bounded device-side wait gave up */
#define LJ_ST_CELL_RANGE 8  /* a particle's cell index was out of range */

/* ---- precision forms ---- */
#define LJ_FP64 0   /* FP64 pair arithmetic, FP64 state and sums */
#define LJ_MIXED 1  /* FP32 pair arithmetic; FP64 positions, velocities and global energy/virial sums */

/* ---- pair-list forms ---- */
#define LJ_LIST_FULL 0  /* every particle lists all partners; force kernel writes without atomics */
#define LJ_LIST_HALF 1  /* each pair once, key = lower index (Sec. 2.4); Newton-3 scatter with atomics */
/* The form chosen per box: the half list in the FP64 form and, in the mixed form, when the full list
 * would hold 75 or more partners per particle ((4/3) pi r_s^3 N / L^3), the full list otherwise.
 * The crossover was measured on GB300 at 16.4M particles, r_s = 3.0: the full list is faster at
 * density 0.5 (56 partners per particle; force 3.04 against 3.91 ms), the half list at density
 * 0.8 (87 partners; 4.60 against 5.26 ms).  ljmd_stats.list_form reports the form in use. */
#define LJ_LIST_AUTO 2

/* ---- list validity rules (Sec. 2.3, Alg. 2) ---- */
#define LJ_VALID_HALF_MARGIN 0     /* rebuild when the largest displacement since the build > margin/2 */
#define LJ_VALID_DUTC 1            /* DUTC: buffer = margin at the build, -= 2 v_max dt per step, rebuild at <= 0 */
#define LJ_VALID_DUTC_LDC 2        /* Alg. 2: DUTC first; when it expires, the large displacement check */
#define LJ_VALID_HALF_MARGIN_LDC 3 /* the margin/2 rule first; when it fires, the large displacement check */

/* ---- truncation of the potential (Sec. 2.1) ---- */
#define LJ_TRUNC_QUADRATIC 0  /* Eq. 2: 4 eps [c2 (r/sigma)^2 + c0] added, V(r_c) = V'(r_c) = 0 */
#define LJ_TRUNC_SHIFT 1      /* c2 = 0, c0 from V(r_c) = 0 (force identical to Eq. 1) */
#define LJ_TRUNC_CUT 2        /* Eq. 1 cut at r_c (c2 = c0 = 0) */

typedef struct ljmd_params {
  double eps;          /* well depth of Eq. 1 */
  double sigma;        /* diameter of Eq. 1 */
  double cutoff;       /* r_c (absolute length), > 0 */
  double margin;       /* r_s - r_c (Sec. 2.3), >= 0 */
  int32_t truncation;  /* LJ_TRUNC_* */
  int32_t list_form;   /* LJ_LIST_FULL, LJ_LIST_HALF or LJ_LIST_AUTO */
  int32_t energy_every; /* inside ljmd_step: evaluate PE and virial every k-th step (0 = only on request) */
  int32_t lanes;       /* threads per key particle in the force kernel: 1,2,4,8,16,32; 0 = tuned default */
} ljmd_params;

typedef struct ljmd_stats {
  int64_t n;               /* particles */
  int64_t steps;           /* velocity-Verlet steps taken since the state was set */
  int64_t rebuilds;        /* pair-list constructions since the state was set */
  int64_t list_entries;    /* entries in the current list (2x the pairs for LJ_LIST_FULL) */
  int64_t cells_per_side;  /* n_g per axis of the cell grid (cell side >= r_s, Sec. 2.2) */
  double box;              /* L */
  double mean_lifetime;    /* steps / rebuilds (list lifetime, Sec. 5.2) */
  double max_displacement; /* largest displacement since the last rebuild, at the last check */
  int32_t status_word;     /* LJ_ST_* bits raised on the device (synchronises) */
  int32_t precision;       /* LJ_FP64 / LJ_MIXED */
  int64_t kernel_launches; /* CUDA kernels this handle has launched */
  int64_t ldc_checks;      /* large displacement checks run (LDC rules) */
  int64_t ldc_kept;        /* of those, checks that kept the list */
  int32_t validity;        /* LJ_VALID_* rule in use */
  int32_t list_form;       /* LJ_LIST_FULL or LJ_LIST_HALF: the form in use (LJ_LIST_AUTO resolved) */
} ljmd_stats;

/* Per-phase device time (CUDA events on the handle's stream), accumulated while profiling is on. */
typedef struct ljmd_profile {
  double force_ms;         /* force kernel (Alg. 4-6) */
  int64_t force_launches;
  double integrate_ms;     /* velocity-Verlet kernel (kick, drift, displacement max, KE) */
  int64_t integrate_launches;
  double rebuild_ms;       /* fold + cell sort + reorder + two-pass list build */
  int64_t rebuilds;
  double energy_ms;        /* final energy reductions */
  int64_t energy_launches;
  double adjoint_ms;       /* adjoint kernel (Hessian-vector product, forces, parameter derivatives) */
  int64_t adjoint_launches;
} ljmd_profile;

typedef struct ljmd_sys ljmd_sys;

/*
 * Create a system handle with potential/list parameters p and precision form
 * (LJ_FP64 or LJ_MIXED).  cuda_stream is a cudaStream_t (NULL = legacy default
 * stream) on the current device; all work of this handle is ordered on it.
 * No particles exist until ljmd_init_lattice or ljmd_set_state.
 * Errors: LJ_EINVAL (NULL out/p, cutoff <= 0, margin < 0, bad enum), LJ_EDEVICE.
 */
int ljmd_create(ljmd_sys** out, const ljmd_params* p, int32_t precision, void* cuda_stream);

/* Free every device and host resource of the handle (NULL is ignored). */
void ljmd_destroy(ljmd_sys* sys);

/*
 * FCC start of the benchmark (Sec. 4.5): M^3 cubic cells of side
 * a = (4/density)^(1/3), four sites per cell, N = 4 M^3, L = M a; particle id
 * order ix, iy, iz, basis site.  Velocities: Gaussian components from the
 * counter-based SplitMix64 stream `seed` (draws 4i..4i+3 of particle i, Box-
 * Muller), mean removed, scaled to sum v^2 = 3 (N - 1) T.  Forces are zero
 * until the next ljmd_compute_forces / ljmd_step.
 * Errors: LJ_EINVAL (M <= 0, density <= 0, T < 0, box too small for the list),
 * LJ_ENOMEM.
 */
int ljmd_init_lattice(ljmd_sys* sys, int64_t cells_per_side, double density, double T, uint64_t seed);

/*
 * Set N particles in a periodic box of side `box`: x[3N] positions (any real
 * values; folded into [0, box) at the next list construction), v[3N]
 * velocities (NULL = zero).  on_device = 0: host arrays; 1: device arrays.
 * Resets step and rebuild counters; the list is rebuilt before the next force.
 * Errors: LJ_EINVAL (n <= 0, box < 2 (r_c + 2 margin), NULL x), LJ_ENOMEM.
 */
int ljmd_set_state(ljmd_sys* sys, int64_t n, double box, const double* x, const double* v, int32_t on_device);

/*
 * Copy the state out in id order: x[3N] (positions as stored: folded into the
 * box at the last list construction, possibly up to margin/2 outside it
 * since), v[3N], f[3N] (forces of the last evaluation).  Any pointer may be
 * NULL.  img (int32 [3N], may be NULL) receives the periodic image counts so
 * that x + img * L is the unwrapped trajectory.  Synchronises the stream.
 */
int ljmd_get_state(ljmd_sys* sys, double* x, double* v, double* f, int32_t* img, int32_t on_device);

/*
 * Construct the pair list (Sec. 2.2-2.4, Alg. 1): fold positions into the
 * box, label particles by cell (cells per side = floor(L / r_s), so the cell
 * side is at least r_s), counting-sort the particles by cell and reorder
 * every particle array in that order (Sec. 3.3), then list every pair with
 * r < r_s = cutoff + margin as a sorted list (KeyPointer / SortedList).  The
 * list is exact: its pair set equals brute force over all pairs with
 * r^2 = dx*dx + dy*dy + dz*dz evaluated in FP64 without FMA.  The cutoff and
 * margin replace those given at creation.  Synchronises once (list size).
 * Errors: LJ_EINVAL (cutoff <= 0, margin < 0, box too small), LJ_ESTATE,
 * LJ_ENOMEM, LJ_ERANGE (more than 2^32 - 1 entries).
 */
int ljmd_build_pairlist(ljmd_sys* sys, double cutoff, double margin);

/*
 * Forces for the current positions over the current list (Alg. 4-6:
 * f = [(24 r^6 - 48)/r^14 + 8 c2] eps/sigma^2 with r in units of sigma, zero
 * for r >= r_c without branching, force on i = f (q_j - q_i)), plus the
 * potential energy (Eq. 2) and virial W = sum_{i<j} r_ij . F_ij.  If no list
 * exists or a particle moved more than margin/2 since it was built, the list
 * is rebuilt first.
 */
int ljmd_compute_forces(ljmd_sys* sys);

/*
 * Advance nsteps of velocity-Verlet (m = 1): v += dt/2 F; x += dt v;
 * F = F(x); v += dt/2 F.  After each drift the largest displacement since
 * the last list construction is reduced on the device; the list is rebuilt
 * whenever it exceeds margin/2 (the two particles of a pair can then have
 * closed in by at most the margin, so every pair with r < r_c is still
 * listed).  Forces must be current on entry (they are computed first if not).
 * Energies are evaluated every params.energy_every steps.
 */
int ljmd_step(ljmd_sys* sys, double dt, int64_t nsteps);

/*
 * Energies of the current state: pe = sum_{i<j} V(r_ij) (Eq. 2), ke = 1/2 sum v^2,
 * virial = sum_{i<j} r_ij . F_ij (FP64 totals).  Evaluates PE/virial first if
 * the stored values are not for the current positions.  Any pointer may be
 * NULL.  Synchronises the stream.
 */
int ljmd_energies(ljmd_sys* sys, double* pe, double* ke, double* virial);

/*
 * Register a device buffer (float64, 4 values per record: step, pe, ke,
 * virial) that ljmd_step fills at every energy evaluation; capacity in
 * records.  NULL disables.  The buffer is caller-owned.  Records past the
 * capacity are dropped.  ljmd_stats().steps tells how far it was filled.
 */
int ljmd_set_energy_log(ljmd_sys* sys, double* device_log, int64_t capacity);

/*
 * The current pair list as unique pairs (i, j), i < j in id order, sorted
 * lexicographically: ij[2k], ij[2k+1] for k < min(cap, npairs).  *npairs
 * receives the number of unique pairs.  Synchronises the stream.
 */
int ljmd_get_pairs(ljmd_sys* sys, int64_t* ij, int64_t cap, int64_t* npairs);

/*
 * Capacity, in list entries (tile padding included), of the static device scratch that
 * ljmd_get_pairs_static uses: 2^19 entries of 8 bytes (4 MiB) per device.
 */
#define LJ_PAIRS_STATIC_MAX_ENTRIES 524288

/*
 * Allocation-free variant of ljmd_get_pairs: the same output (unique pairs (i, j), i < j in id
 * order, sorted lexicographically; the first min(cap, npairs) of them in ij[2k], ij[2k+1];
 * *npairs = the number of unique pairs) for lists of at most LJ_PAIRS_STATIC_MAX_ENTRIES
 * entries.  It has no counterpart in the paper; it exists so that the list can be exported
 * repeatedly (e.g. checked inside a long run) without the per-call device buffer of
 * ljmd_get_pairs.
 *
 * It allocates nothing: the list is decoded into a file-scope static device array of
 * LJ_PAIRS_STATIC_MAX_ENTRIES 64-bit slots plus a 256-byte header, turned into 64-bit keys
 * (i << 32 | j), sorted on the device and copied into ij.  Each call clears what must start
 * cleared: the kept-pair counter (to zero) and the key slots it uses (to all ones).
 *  - The first call on a device resolves the scratch's address (cudaGetSymbolAddress, which may
 *    load the module); make that first call before any stream capture.  Later calls on the
 *    device reuse the address.
 *  - One scratch per device is shared by every handle and stream of the process: calls that
 *    overlap on one device (from two threads, or on two streams before either completes) race
 *    and give wrong pairs.  Serialise them.
 *  - The list must exist (ljmd_build_pairlist, ljmd_compute_forces or ljmd_step made it):
 *    constructing one may allocate, so this call never does.
 *  - The handle's device must be the current device.
 *  - Synchronises the stream.
 * Errors: LJ_EINVAL (NULL sys/npairs, cap < 0, ij NULL with cap > 0, another device current),
 * LJ_ESTATE (no particles or no list), LJ_ERANGE (the list has more than
 * LJ_PAIRS_STATIC_MAX_ENTRIES entries; a line naming both sizes goes to stderr and nothing is
 * written), LJ_EDEVICE (a CUDA error, or the device status word was raised, e.g. by a list entry
 * that decodes out of range: ij and *npairs are then left unwritten, as by ljmd_get_pairs).
 */
int ljmd_get_pairs_static(ljmd_sys* sys, int64_t* ij, int64_t cap, int64_t* npairs);

/*
 * Budget of the bounded device-side waits, in SM clock cycles, for every system and batch of
 * the process on the current device (0 restores the default of 4e9 cycles, about 2 s).  No
 * counterpart in the paper: the waits are those of the staged tiles of the list, force and
 * adjoint kernels (a tile's bulk copies) and of the pipelined force kernel (producer and
 * consumer warps waiting for each other).  A wait that exceeds the budget records LJ_ST_TIMEOUT
 * in the device status word and its CTA leaves after the copies it issued have landed (those
 * final waits keep the default budget), so the call returns LJ_EDEVICE and the device stays
 * usable.  A budget below the default also stops the waits from suspending, so a small budget
 * makes them give up before their copies land: a test of the timeout paths.  Synchronises the
 * device.  Errors: LJ_EINVAL (cycles < 0), LJ_EDEVICE (CUDA error).
 */
int ljmd_set_wait_budget(int64_t cycles);

/*
 * Adjoint pass at the current positions over the current list (the list is built first if there
 * is none): hw = H(x) w, the Hessian of the potential energy (Eq. 2 summed over pairs with
 * r < r_c) times w, from the pair energy u(s) as a function of s = r^2:
 *   (H w)_i = sum_j [2 u'(s) (w_i - w_j) + 4 u''(s) d (d . (w_i - w_j))],  d = x_j - x_i.
 * The force Jacobian is -H.  dtheta (4 doubles, may be NULL) receives w . dF/deps,
 * w . dF/dsigma, dPE/deps and dPE/dsigma, with r_c = (cutoff / sigma) sigma scaling with sigma
 * (the truncation constants c2, c0 of Eq. 2 stay fixed).  w and hw are 3N FP64 in id order, host
 * (on_device = 0) or device (1).  The paper has no adjoint; this differentiates its pair force.
 * Mixed form: FP32 pair arithmetic, FP64 results.  Synchronises the stream.
 * The adjoint needs the full list: a handle created with LJ_LIST_HALF gets LJ_ESTATE, and one
 * created with LJ_LIST_AUTO uses the full list from this call on.
 * Errors: LJ_EINVAL (NULL w or hw), LJ_ESTATE (no particles, or an LJ_LIST_HALF handle),
 * LJ_ENOMEM, LJ_EDEVICE.
 */
int ljmd_hvp(ljmd_sys* sys, const double* w, double* hw, double* dtheta, int32_t on_device);

/*
 * Differentiable trajectory: from (x0, v0) (n particles, box side `box`, 3n FP64 each, id order,
 * x0 unwrapped) run nsteps of velocity-Verlet (Sec. 4.5) with step dt and return
 *   *loss = (1 / n_pe) sum_{t > nsteps - n_pe} PE(x_t) / n  +  (1 / n) sum_i |x_i(nsteps) - x_i(0)|^2
 * (unwrapped positions), and, if any of gx0, gv0, gtheta is non-NULL, its gradients with respect
 * to x0, v0 (3n FP64 each) and (eps, sigma) (gtheta[2]).  The gradients come from the reverse-time
 * recurrences of velocity-Verlet with h = dt / 2 (one adjoint pass, i.e. one Hessian-vector
 * product, per state), recomputing the states of each segment of ckpt_every steps from a
 * checkpoint stored in the forward run.  Arrays are host (on_device = 0) or device (1).  The
 * handle's state is replaced: it ends at the positions x0, velocities unspecified; the energy log
 * registered with ljmd_set_energy_log receives nothing from this call.  The paper has no
 * adjoint; this differentiates its integrator and pair force.  Synchronises the stream.
 * Like ljmd_hvp it needs the full list (LJ_LIST_HALF: LJ_ESTATE; LJ_LIST_AUTO: full from now on).
 * Errors: LJ_EINVAL (n <= 0, nsteps < 1, n_pe outside [0, nsteps], ckpt_every < 1, NULL x0, v0 or
 * loss, box too small), LJ_ESTATE (an LJ_LIST_HALF handle), LJ_ENOMEM, LJ_EDEVICE.
 */
int ljmd_traj_loss_grad(ljmd_sys* sys, int64_t n, double box, const double* x0, const double* v0, double dt,
                        int64_t nsteps, int64_t n_pe, int64_t ckpt_every, double* loss, double* gx0, double* gv0,
                        double* gtheta, int32_t on_device);

/*
 * The cell grid of the last list construction (Sec. 2.2, Fig. 3), read only: the particles were
 * folded into the box, labelled c = (cx n + cy) n + cz with ck = floor(x_k n / L) (n cells per
 * side), counting-sorted by label with ties in id order, and every particle array was reordered
 * that way (Sec. 3.3).  grid_pointer[c] (c <= n^3, the first min(pointer_cap, n^3 + 1) values) is
 * GridPointer, the position of cell c's first particle in that order (grid_pointer[n^3] = N);
 * grid_list[k] (the first min(list_cap, N) values) is GridList, the id of the particle in
 * position k.  *ncells receives n^3.  Caller-owned host arrays; synchronises the stream.
 * Errors: LJ_EINVAL (NULL sys or ncells, negative capacity, NULL array with a positive capacity),
 * LJ_ESTATE (no particles or no list yet), LJ_EDEVICE.
 */
int ljmd_get_grid(ljmd_sys* sys, int64_t* grid_pointer, int64_t pointer_cap, int64_t* grid_list, int64_t list_cap,
                  int64_t* ncells);

/* Counters and state of the handle (synchronises the stream). */
int ljmd_get_stats(ljmd_sys* sys, ljmd_stats* out);

/*
 * Turn per-phase timing on (enable = 1, resets the accumulators) or off (0).  While on, CUDA
 * events are recorded on the handle's stream around every force, integrate, rebuild, energy and
 * adjoint launch; the kernels themselves are unchanged.
 */
int ljmd_set_profiling(ljmd_sys* sys, int32_t enable);

/* Accumulated per-phase device times since profiling was enabled (synchronises the stream). */
int ljmd_get_profile(ljmd_sys* sys, ljmd_profile* out);

/*
 * Kernel shape of the list and force kernels (the autotuner's knobs); 0 keeps the default.
 * tile_cells: cells per shared-memory tile along z (1..14; default: for the mixed form with the
 * full list about 165 particles per tile, at most 12 cells, else 4); lanes: threads per key
 * particle in the force kernel (1, 2, 4, 8, 16, 32; default: for the mixed form with the full list
 * 2 for tiles of 96 or more particles, else 4); force_ctas_per_sm: resident force CTAs per SM
 * (1..4; the pipelined kernel takes as many as fit); force_buffers: tile buffers per force CTA
 * (1: tiles staged one after the other; 2: the next tile's copies overlap the current tile's
 * arithmetic; for the mixed form with the full list and the FP64 form with the half list this is
 * the pipelined kernel, in which producer warps stage tiles and consumer warps compute, and it is
 * the default there; 1 is the default otherwise).  A new tile_cells or force_buffers
 * takes effect at the next list construction (forced at the next force evaluation).  Results
 * do not depend on these knobs beyond FP32 summation order.
 */
int ljmd_set_tuning(ljmd_sys* sys, int32_t tile_cells, int32_t lanes, int32_t force_ctas_per_sm,
                    int32_t force_buffers);

/* ---- batched replicas ------------------------------------------------------------------- */

/*
 * Many independent periodic LJ systems (replicas) of uneven size, density and temperature,
 * advanced together with the same method (mixed form, full list): every phase of the step is one
 * launch over all replicas, the list-validity rule (rebuild when the largest displacement of any
 * replica exceeds margin/2) is evaluated on the device, and K steps can be captured once as a
 * CUDA graph and replayed.  Replica r owns particles [base_r, base_r + n[r]) of every array, with
 * base_r = n[0] + ... + n[r-1]; all arrays are in that concatenated order.  The paper treats one
 * system; batching is this library's extension of the same per-system method.
 */
typedef struct ljmd_batch ljmd_batch;

typedef struct ljmd_batch_stats {
  int64_t replicas;        /* R */
  int64_t n;               /* particles over all replicas */
  int64_t steps;           /* steps since the state was set */
  int64_t rebuilds;        /* list constructions (host-driven and device-decided) */
  int64_t list_entries;    /* entries of the current lists, all replicas */
  int64_t tiles;           /* shared-memory tiles over all replicas */
  int64_t cells;           /* cells over all replicas */
  int64_t kernel_launches; /* kernels launched (graph replays count their kernels) */
  int32_t status_word;     /* LJ_ST_* bits raised on the device */
  int32_t tile_cells;      /* preferred cells per tile along z */
  int32_t lanes;           /* threads per key particle in the force kernel */
  int32_t pad;
} ljmd_batch_stats;

/*
 * Create a batch of `replicas` systems with common potential and list parameters p (cutoff,
 * margin, eps, sigma, truncation; list_form is full; p->lanes 2, 4 or 8 or 0 for the default)
 * and per-replica particle counts n[r] and box sides box[r] (host arrays).  Every box needs
 * L >= 2 (r_s + margin); boxes under 3 r_s have 2 cells per side, whose tiles stage aliased
 * neighbour cells under both periodic images (at most one of which is ever within r_s + margin of
 * a key, so the lists stay exact).  The batch works on its own
 * stream; every call first waits for the work queued so far on cuda_stream (a cudaStream_t, NULL =
 * legacy default stream).  Errors: LJ_EINVAL (a box under 2 (r_s + margin)), LJ_ERANGE (more than
 * 2^32 - 1 cells, more than 10^9 particles), LJ_ENOMEM, LJ_EDEVICE.
 */
int ljmd_batch_create(ljmd_batch** out, const ljmd_params* p, int32_t replicas, const int64_t* n, const double* box,
                      void* cuda_stream);

/* Free every resource of the batch (NULL is ignored). */
void ljmd_batch_destroy(ljmd_batch* b);

/*
 * Set all replicas' states: x[3 i + k] positions (folded into the replica's box), v velocities
 * (NULL = 0), i over the concatenated particles; host (on_device = 0) or device arrays.  The
 * lists are rebuilt (with capacities sized for the following steps) before the next force.
 */
int ljmd_batch_set_state(ljmd_batch* b, const double* x, const double* v, int32_t on_device);

/*
 * Advance every replica nsteps velocity-Verlet steps (Sec. 4.5) with step dt.  graph_steps = K > 0:
 * the K-step sequence (kick-drift with displacement check, device-decided rebuild, force; final
 * kick) is captured once as a CUDA graph (re-captured when dt or K changes) and replayed
 * floor(nsteps / K) times, the rest run as plain launches; K = 0: plain launches.  No host
 * synchronisation between steps; synchronises once at the end.  Capacities of the lists are fixed
 * at the last host construction (with headroom); if a device-side construction exceeds them the
 * status word is raised and LJ_EDEVICE is returned (set the state again to resize).
 */
int ljmd_batch_step(ljmd_batch* b, double dt, int64_t nsteps, int32_t graph_steps);

/* Per-replica PE (Eq. 2), kinetic energy and virial of the current state (host arrays of R). */
int ljmd_batch_energies(ljmd_batch* b, double* pe, double* ke, double* virial);

/* Positions (as stored, folded at the last construction), velocities and forces in the
 * concatenated caller order; any pointer may be NULL.  Synchronises. */
int ljmd_batch_get_state(ljmd_batch* b, double* x, double* v, double* f, int32_t on_device);

/* Unique pairs (i, j), i < j, of replica r's current list in its own particle numbering, sorted;
 * as ljmd_get_pairs.  Synchronises. */
int ljmd_batch_get_pairs(ljmd_batch* b, int32_t replica, int64_t* ij, int64_t cap, int64_t* npairs);

int ljmd_batch_get_stats(ljmd_batch* b, ljmd_batch_stats* out);

/* Kernel shape: tile_cells (1..14, 0 keeps) and force lanes (2, 4, 8; 0 keeps).  Drops the graph. */
int ljmd_batch_set_tuning(ljmd_batch* b, int32_t tile_cells, int32_t lanes);

/*
 * Autotuner: for tile_cells in {2, 3, 4, 6} and lanes in {2, 4, 8}, construct the lists at the
 * current positions and time `trials` force launches and the construction (CUDA events); keep the
 * shape with the least force + construction / 10.  The state is unchanged.  Outputs may be NULL.
 */
int ljmd_batch_autotune(ljmd_batch* b, int32_t trials, int32_t* best_tile, int32_t* best_lanes, double* best_ms);

/*
 * Mean device time, in milliseconds, of one force launch over all replicas (the kernel of Alg. 4-6
 * on every replica's list at the current positions): one warm-up launch, then `trials` launches
 * timed with CUDA events on the batch's stream.  The forces are recomputed; positions, velocities
 * and lists are unchanged.  A measurement call (no counterpart in the paper), for the roofline of
 * the batched form.  Synchronises.  Errors: LJ_EINVAL (NULL b or ms_per_launch, trials <= 0),
 * LJ_ESTATE (no state set), LJ_EDEVICE.
 */
int ljmd_batch_time_force(ljmd_batch* b, int32_t trials, double* ms_per_launch);

/*
 * List-validity rule (Sec. 2.3, Alg. 2); the list is rebuilt when the rule says it expired.
 *  LJ_VALID_HALF_MARGIN (default): the largest displacement since the build exceeds margin/2.
 *  LJ_VALID_DUTC: the dynamical upper time cutoff, buffer_length = margin at the build, reduced by
 *    2 v_max dt every step (v_max: largest drift speed of the step), expired at <= 0.
 *  LJ_VALID_DUTC_LDC: Alg. 2: when DUTC expires, the large displacement check (LDC) decides: the
 *    particles that moved more than margin - (largest displacement) form L_D; the list is kept if
 *    |L_D| <= max_ld (N_l) and no pair of L_D is unlisted yet closer than r_c now.  Rerun every
 *    step until it fails.
 *  LJ_VALID_HALF_MARGIN_LDC: the margin/2 rule first, then the LDC as above.
 * max_ld: N_l (0 keeps the current, default 4096).  A new rule takes effect at the next list
 * construction (forced at the next force evaluation).  Errors: LJ_EINVAL.
 */
int ljmd_set_validity(ljmd_sys* sys, int32_t mode, int32_t max_ld);

/* Human-readable name of a status code. */
const char* ljmd_strerror(int code);

/* Library version, major * 10000 + minor * 100 + patch. */
int ljmd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LJMD_H */
