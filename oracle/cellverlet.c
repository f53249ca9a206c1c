/*
 * cellverlet.c -- the paper's method on the CPU in FP64: a CPU baseline, not the oracle.
 *
 * TEST AND BENCHMARK INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
 * Python binding) may include, link or call this file; it shares no code with that path or with
 * ljoracle.c.  bench.py times it as the CPU baseline of the Verlet-list method on the host cores,
 * and tests/ check it against the all-pairs oracle.
 *
 * One velocity-Verlet step (second-order symplectic, Sec. 4.5) over a bookkeeping pair list
 * (Sec. 2.3): the list holds every pair closer than the search length r_s = r_c + margin and is
 * rebuilt when a particle has moved more than margin/2 since the last construction.  A
 * construction (Sec. 2.2-2.4, Alg. 1, Fig. 3, Fig. 6):
 *   1. fold the positions into [0, L) (image counts kept, so unwrapped positions come back out);
 *   2. label each particle by its cell, c = (cx n + cy) n + cz, n = floor(L / r_s) cells per side;
 *   3. counting sort by label (GridParticleNumber, GridPointer, GridList), ties in the current
 *      order, and reorder every particle array in that order (the sort of Sec. 3.3, here at every
 *      construction);
 *   4. for every key i, the partners j > i in i's cell and the 26 neighbour cells with
 *      r^2 = dx*dx + dy*dy + dz*dz < r_s^2 (min image), stored as KeyPointer / SortedList
 *      (Sec. 2.4: each pair once, the key being the lower index).  With fewer than 3 cells per
 *      side the neighbour cells repeat, so every j > i is tested instead.
 * The force (Alg. 4-6): for each key, the sum over its partners of f (q_j - q_i) with
 *   f = (eps / sigma^2) [ (24 s^3 - 48) / s^7 + 8 c2 ],  s = r^2 / sigma^2,
 * set to zero for r >= r_c by a select instead of a branch (Alg. 5) and one division per pair
 * (Alg. 6); Newton's third law adds -f (q_j - q_i) to j.  Threads (OpenMP) take contiguous key
 * ranges and scatter into private force arrays that are summed in a fixed order afterwards, so
 * results do not depend on timing.  PE (Eq. 2) and the virial W = sum_{i<j} r_ij . F_ij are
 * summed alongside.
 *
 * Layout: positions, velocities and forces AoS [3 i + k], FP64.  Reduced units, m = 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int64_t n;
  double L, rs2, rc2, half_margin;
  double eps, sig2, c2, c0;
  int64_t nc, ncells;     /* cells per side, cells */
  double *x, *v, *f;      /* sorted order */
  double* xref;           /* positions at the last construction */
  int64_t* id;            /* sorted position -> caller id */
  int32_t* img;           /* periodic image counts, sorted order */
  int64_t* cell;          /* cell label of each particle */
  int64_t* gptr;          /* GridPointer [ncells + 1] */
  int64_t* kp;            /* KeyPointer [n + 1] */
  int32_t* sl;            /* SortedList */
  int64_t sl_cap;
  int nthreads;
  double* fpriv;          /* per-thread force arrays [nthreads][3 n] */
  int64_t rebuilds;
} cv_sys;

static double now_s(void) {
#ifdef _OPENMP
  return omp_get_wtime();
#else
  return 0.0;
#endif
}

static int threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static int thread_id(void) {
#ifdef _OPENMP
  return omp_get_thread_num();
#else
  return 0;
#endif
}

static double wrap_d(double d, double L) {
  if (d > 0.5 * L) return d - L;
  if (d < -0.5 * L) return d + L;
  return d;
}

/* Steps 1-3: fold, label, stable counting sort, reorder. */
static int sort_by_cell(cv_sys* s) {
  const int64_t n = s->n, nc = s->nc, ncells = s->ncells;
  const double L = s->L, inv_h = (double)nc / L;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t c[3];
    for (int k = 0; k < 3; ++k) {
      double q = s->x[3 * i + k];
      if (q >= L) {
        q -= L;
        s->img[3 * i + k] += 1;
      } else if (q < 0.0) {
        q += L;
        s->img[3 * i + k] -= 1;
      }
      s->x[3 * i + k] = q;
      int64_t ck = (int64_t)floor(q * inv_h);
      c[k] = ck < 0 ? 0 : (ck >= nc ? nc - 1 : ck);
    }
    s->cell[i] = (c[0] * nc + c[1]) * nc + c[2];
  }
  /* counting sort, stable: per-thread histograms over contiguous chunks, prefix over (cell, thread) */
  const int T = s->nthreads;
  int64_t* hist = (int64_t*)calloc((size_t)T * (size_t)ncells, sizeof(int64_t));
  int64_t* perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!hist || !perm) {
    free(hist);
    free(perm);
    return -1;
  }
#pragma omp parallel num_threads(T)
  {
    const int t = thread_id();
    const int64_t a = n * t / T, b = n * (t + 1) / T;
    int64_t* h = hist + (size_t)t * (size_t)ncells;
    for (int64_t i = a; i < b; ++i) h[s->cell[i]] += 1;
  }
  int64_t run = 0;
  for (int64_t c = 0; c < ncells; ++c) {
    s->gptr[c] = run;
    for (int t = 0; t < T; ++t) {
      const int64_t cnt = hist[(size_t)t * (size_t)ncells + c];
      hist[(size_t)t * (size_t)ncells + c] = run;
      run += cnt;
    }
  }
  s->gptr[ncells] = run;
#pragma omp parallel num_threads(T)
  {
    const int t = thread_id();
    const int64_t a = n * t / T, b = n * (t + 1) / T;
    int64_t* h = hist + (size_t)t * (size_t)ncells;
    for (int64_t i = a; i < b; ++i) perm[h[s->cell[i]]++] = i;
  }
  free(hist);
  /* reorder every particle array through a staging buffer */
  double* tmp = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  int64_t* tid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int32_t* timg = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(n > 0 ? n : 1));
  if (!tmp || !tid || !timg) {
    free(tmp);
    free(tid);
    free(timg);
    free(perm);
    return -1;
  }
  double* arrs[3] = {s->x, s->v, s->f};
  for (int a = 0; a < 3; ++a) {
    double* A = arrs[a];
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k)
      for (int q = 0; q < 3; ++q) tmp[3 * k + q] = A[3 * perm[k] + q];
    memcpy(A, tmp, sizeof(double) * 3 * (size_t)n);
  }
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < n; ++k) {
    tid[k] = s->id[perm[k]];
    for (int q = 0; q < 3; ++q) timg[3 * k + q] = s->img[3 * perm[k] + q];
  }
  memcpy(s->id, tid, sizeof(int64_t) * (size_t)n);
  memcpy(s->img, timg, sizeof(int32_t) * 3 * (size_t)n);
  free(tmp);
  free(tid);
  free(timg);
  free(perm);
  /* labels in the new order follow from the grid pointers */
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < ncells; ++c)
    for (int64_t k = s->gptr[c]; k < s->gptr[c + 1]; ++k) s->cell[k] = c;
  return 0;
}

static int pair_in(const cv_sys* s, int64_t i, int64_t j) {
  const double* xi = s->x + 3 * i;
  const double* xj = s->x + 3 * j;
  const double dx = wrap_d(xj[0] - xi[0], s->L), dy = wrap_d(xj[1] - xi[1], s->L), dz = wrap_d(xj[2] - xi[2], s->L);
  const double r2 = dx * dx + dy * dy + dz * dz;
  return r2 < s->rs2;
}

/* Partners j > i of key i (Alg. 1): counted (out == NULL) or written. */
static int64_t key_partners(const cv_sys* s, int64_t i, int32_t* out) {
  int64_t m = 0;
  const int64_t nc = s->nc;
  if (nc < 3) {
    for (int64_t j = i + 1; j < s->n; ++j)
      if (pair_in(s, i, j)) {
        if (out) out[m] = (int32_t)j;
        ++m;
      }
    return m;
  }
  const int64_t c = s->cell[i];
  const int64_t cx = c / (nc * nc), cy = (c / nc) % nc, cz = c % nc;
  /* neighbour cells in ascending label order, so that each key's partners come out sorted */
  int64_t nb[27];
  int cnt = 0;
  for (int a = -1; a <= 1; ++a)
    for (int b = -1; b <= 1; ++b)
      for (int d = -1; d <= 1; ++d) {
        const int64_t X = (cx + a + nc) % nc, Y = (cy + b + nc) % nc, Z = (cz + d + nc) % nc;
        const int64_t q = (X * nc + Y) * nc + Z;
        if (q >= c) nb[cnt++] = q;
      }
  for (int u = 1; u < cnt; ++u) { /* insertion sort of at most 27 labels */
    const int64_t key = nb[u];
    int w = u;
    while (w > 0 && nb[w - 1] > key) {
      nb[w] = nb[w - 1];
      --w;
    }
    nb[w] = key;
  }
  for (int u = 0; u < cnt; ++u) {
    const int64_t q = nb[u];
    int64_t j0 = s->gptr[q];
    if (q == c) j0 = i + 1;
    for (int64_t j = j0; j < s->gptr[q + 1]; ++j)
      if (pair_in(s, i, j)) {
        if (out) out[m] = (int32_t)j;
        ++m;
      }
  }
  return m;
}

static int build_list(cv_sys* s) {
  s->rebuilds += 1;
  if (sort_by_cell(s)) return -1;
  const int64_t n = s->n;
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; ++i) s->kp[i + 1] = key_partners(s, i, NULL);
  s->kp[0] = 0;
  for (int64_t i = 0; i < n; ++i) s->kp[i + 1] += s->kp[i];
  const int64_t P = s->kp[n];
  if (P > s->sl_cap) {
    free(s->sl);
    s->sl_cap = P + P / 4 + 1024;
    s->sl = (int32_t*)malloc(sizeof(int32_t) * (size_t)s->sl_cap);
    if (!s->sl) return -1;
  }
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; ++i) key_partners(s, i, s->sl + s->kp[i]);
  memcpy(s->xref, s->x, sizeof(double) * 3 * (size_t)n);
  return 0;
}

/* Alg. 4-6 over the half list; PE and virial returned through pe, vir. */
static void compute_forces(cv_sys* s, double* pe, double* vir) {
  const int64_t n = s->n;
  const int T = s->nthreads;
  const double L = s->L, rc2 = s->rc2, sig2 = s->sig2, eps = s->eps;
  const double fpre = eps / sig2, f8c2 = 8.0 * s->c2, e4 = 4.0 * eps, c2 = s->c2, c0 = s->c0;
  double pe_t = 0.0, vir_t = 0.0;
#pragma omp parallel num_threads(T) reduction(+ : pe_t, vir_t)
  {
    const int t = thread_id();
    double* F = s->fpriv + (size_t)t * 3 * (size_t)n;
    memset(F, 0, sizeof(double) * 3 * (size_t)n);
    const int64_t a = n * t / T, b = n * (t + 1) / T;
    for (int64_t i = a; i < b; ++i) {
      const double xi = s->x[3 * i], yi = s->x[3 * i + 1], zi = s->x[3 * i + 2];
      double fx = 0.0, fy = 0.0, fz = 0.0;
      for (int64_t e = s->kp[i]; e < s->kp[i + 1]; ++e) {
        const int64_t j = s->sl[e];
        const double dx = wrap_d(s->x[3 * j] - xi, L), dy = wrap_d(s->x[3 * j + 1] - yi, L),
                     dz = wrap_d(s->x[3 * j + 2] - zi, L);
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double si = sig2 / r2; /* the one division of the pair (Alg. 6) */
        const double s3i = si * si * si;
        double ff = fpre * (si * s3i * (24.0 - 48.0 * s3i) + f8c2);
        double vv = e4 * (s3i * s3i - s3i + c2 * (r2 / sig2) + c0);
        const int in = r2 < rc2;
        ff = in ? ff : 0.0; /* Alg. 5: select, no branch */
        vv = in ? vv : 0.0;
        fx += ff * dx;
        fy += ff * dy;
        fz += ff * dz;
        F[3 * j] -= ff * dx;
        F[3 * j + 1] -= ff * dy;
        F[3 * j + 2] -= ff * dz;
        pe_t += vv;
        vir_t += -ff * r2;
      }
      F[3 * i] += fx;
      F[3 * i + 1] += fy;
      F[3 * i + 2] += fz;
    }
  }
  /* fixed-order sum of the private arrays */
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < 3 * n; ++q) {
    double acc = 0.0;
    for (int t = 0; t < T; ++t) acc += s->fpriv[(size_t)t * 3 * (size_t)n + q];
    s->f[q] = acc;
  }
  *pe = pe_t;
  *vir = vir_t;
}

static double max_disp2(const cv_sys* s) {
  double m = 0.0;
  const int64_t n = s->n;
#pragma omp parallel for schedule(static) reduction(max : m)
  for (int64_t i = 0; i < n; ++i) {
    const double dx = s->x[3 * i] - s->xref[3 * i], dy = s->x[3 * i + 1] - s->xref[3 * i + 1],
                 dz = s->x[3 * i + 2] - s->xref[3 * i + 2];
    const double d2 = dx * dx + dy * dy + dz * dz;
    if (d2 > m) m = d2;
  }
  return m;
}

static void cv_free(cv_sys* s) {
  free(s->x);
  free(s->v);
  free(s->f);
  free(s->xref);
  free(s->id);
  free(s->img);
  free(s->cell);
  free(s->gptr);
  free(s->kp);
  free(s->sl);
  free(s->fpriv);
}

/*
 * Run nsteps of velocity-Verlet with the Verlet-list method from positions x and velocities v
 * (n particles, id order, any real positions; v may be NULL for zero).  On return x holds the
 * unwrapped positions, v the velocities, f (may be NULL) the forces, all in id order; pe, ke, vir
 * the energies of the final state (Eq. 2 summed over pairs, 1/2 sum v^2, sum r . F); rebuilds the
 * constructions (the first included); seconds the wall time of the nsteps (the first
 * construction and force excluded).  nsteps = 0 evaluates the forces of x.  Returns 0, or -1 if
 * memory ran out, -2 for a box under 2 r_s.
 */
int cv_run(int64_t n, double* x, double* v, double L, double rc, double margin, double eps, double sigma, double c2,
           double c0, double dt, int64_t nsteps, double* f, double* pe, double* ke, double* vir, int64_t* rebuilds,
           int64_t* list_pairs, double* seconds) {
  const double rs = rc + margin;
  if (!(L >= 2.0 * rs)) return -2;
  cv_sys s;
  memset(&s, 0, sizeof(s));
  s.n = n;
  s.L = L;
  s.rs2 = rs * rs;
  s.rc2 = rc * rc;
  s.half_margin = 0.5 * margin;
  s.eps = eps;
  s.sig2 = sigma * sigma;
  s.c2 = c2;
  s.c0 = c0;
  s.nc = (int64_t)floor(L / rs);
  if (s.nc < 1) s.nc = 1;
  s.ncells = s.nc * s.nc * s.nc;
  s.nthreads = threads();
  const size_t n3 = 3 * (size_t)(n > 0 ? n : 1);
  s.x = (double*)malloc(sizeof(double) * n3);
  s.v = (double*)calloc(n3, sizeof(double));
  s.f = (double*)calloc(n3, sizeof(double));
  s.xref = (double*)malloc(sizeof(double) * n3);
  s.id = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  s.img = (int32_t*)calloc(n3, sizeof(int32_t));
  s.cell = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  s.gptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s.ncells + 1));
  s.kp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  s.fpriv = (double*)malloc(sizeof(double) * n3 * (size_t)s.nthreads);
  if (!s.x || !s.v || !s.f || !s.xref || !s.id || !s.img || !s.cell || !s.gptr || !s.kp || !s.fpriv) {
    cv_free(&s);
    return -1;
  }
  memcpy(s.x, x, sizeof(double) * 3 * (size_t)n);
  if (v) memcpy(s.v, v, sizeof(double) * 3 * (size_t)n);
  for (int64_t i = 0; i < n; ++i) s.id[i] = i;
  double p = 0.0, w = 0.0;
  if (build_list(&s)) {
    cv_free(&s);
    return -1;
  }
  compute_forces(&s, &p, &w);
  const double h = 0.5 * dt, lim2 = s.half_margin * s.half_margin;
  const double t0 = now_s();
  for (int64_t step = 0; step < nsteps; ++step) {
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < 3 * n; ++q) {
      s.v[q] += h * s.f[q];
      s.x[q] += dt * s.v[q];
    }
    if (max_disp2(&s) > lim2 && build_list(&s)) {
      cv_free(&s);
      return -1;
    }
    compute_forces(&s, &p, &w);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < 3 * n; ++q) s.v[q] += h * s.f[q];
  }
  if (seconds) *seconds = now_s() - t0;
  double k = 0.0;
  for (int64_t q = 0; q < 3 * n; ++q) k += s.v[q] * s.v[q];
  /* back to id order, positions unwrapped */
  for (int64_t i = 0; i < n; ++i) {
    const int64_t o = s.id[i];
    for (int q = 0; q < 3; ++q) {
      x[3 * o + q] = s.x[3 * i + q] + (double)s.img[3 * i + q] * L;
      if (v) v[3 * o + q] = s.v[3 * i + q];
      if (f) f[3 * o + q] = s.f[3 * i + q];
    }
  }
  if (pe) *pe = p;
  if (ke) *ke = 0.5 * k;
  if (vir) *vir = w;
  if (rebuilds) *rebuilds = s.rebuilds;
  if (list_pairs) *list_pairs = s.kp[n];
  cv_free(&s);
  return 0;
}
