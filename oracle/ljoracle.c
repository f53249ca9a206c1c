/*
 * ljoracle.c -- plain FP64 CPU oracle for the Lennard-Jones MD hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library
 * and its Python binding) may include, link or call this file.  It is used by
 * tests/, by __graft_entry__.smoke() and by the CPU-baseline leg of bench.py.
 *
 * Everything here is the plain definition of what the method computes, in
 * double precision, O(N^2) over all pairs, with no cell grid, no pair list,
 * no blocking and no reordering.  The Verlet-list method of the paper reaches
 * exactly these results (up to summation order) as long as its list is valid
 * (Sec. 2.3, the bookkeeping method), so the all-pairs sum is the oracle.
 *
 * Compile with -ffp-contract=off: the pair-set distance r^2 = dx*dx+dy*dy+dz*dz
 * must be evaluated without FMA contraction so that both sides agree bit for
 * bit on which pairs lie within the search length.
 *
 * Conventions (reduced units, m = 1):
 *   positions x[3*i+k], velocities v[3*i+k], forces F[3*i+k]  (AoS, FP64)
 *   min image per component: d > L/2 -> d -= L ; d < -L/2 -> d += L
 *   force on i from j:  F_ij = f(r) * (q_j - q_i)   (Alg. 6)
 *   with f = (eps/sigma^2) * [ (24 s^3 - 48) / s^7 + 8 c2 ],  s = r^2/sigma^2
 *   pair potential (Eq. 2): V = 4 eps [ s^-6 - s^-3 + c2 s + c0 ]  for r < rc
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Truncation schemes of Sec. 2.1. */
enum {
  OR_TRUNC_QUADRATIC = 0, /* Eq. 2: c2 (r/sigma)^2 + c0, V(rc) = V'(rc) = 0 */
  OR_TRUNC_SHIFT = 1,     /* c2 = 0 and c0 chosen so that V(rc) = 0        */
  OR_TRUNC_CUT = 2,       /* c2 = c0 = 0: Eq. 1 cut at rc                  */
};

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/*
 * Coefficients of the additive truncation terms, Eq. 2 (Sec. 2.1).
 * With x = rc/sigma the two conditions V(rc) = 0 and V'(rc) = 0 read
 *   x^-12 - x^-6 + c2 x^2 + c0 = 0
 *   -12 x^-13 + 6 x^-7 + 2 c2 x = 0
 * whose solution is c2 = 6 x^-14 - 3 x^-8 and c0 = -7 x^-12 + 4 x^-6.
 * The constant-shift variant (c2 = 0) only asks V(rc) = 0: c0 = x^-6 - x^-12.
 */
void or_trunc_coeffs(double x, int mode, double* c2, double* c0) {
  double x2 = x * x, x6 = x2 * x2 * x2, x8 = x6 * x2, x12 = x6 * x6, x14 = x12 * x2;
  if (mode == OR_TRUNC_QUADRATIC) {
    *c2 = 6.0 / x14 - 3.0 / x8;
    *c0 = -7.0 / x12 + 4.0 / x6;
  } else if (mode == OR_TRUNC_SHIFT) {
    *c2 = 0.0;
    *c0 = 1.0 / x6 - 1.0 / x12;
  } else {
    *c2 = 0.0;
    *c0 = 0.0;
  }
}

/* Eq. 1, the untruncated potential, V(r) = 4 eps [ (sigma/r)^12 - (sigma/r)^6 ]. */
double or_v_raw(double r, double eps, double sigma) {
  double sr = sigma / r, sr6 = pow(sr, 6.0);
  return 4.0 * eps * (sr6 * sr6 - sr6);
}

/* -dV/dr of Eq. 1 (radial force, positive = repulsive). */
double or_f_raw(double r, double eps, double sigma) {
  double sr = sigma / r, sr6 = pow(sr, 6.0);
  return 4.0 * eps * (12.0 * sr6 * sr6 - 6.0 * sr6) / r;
}

/* Eq. 2 pair potential for r^2 (zero at and beyond rc). */
double or_pair_v(double r2, double eps, double sigma, double rc, double c2, double c0) {
  if (r2 >= rc * rc) return 0.0;
  double s = r2 / (sigma * sigma);
  double s3 = s * s * s, s6 = s3 * s3;
  return 4.0 * eps * (1.0 / s6 - 1.0 / s3 + c2 * s + c0);
}

/* Alg. 6 force coefficient: the force on i from j is f * (q_j - q_i). */
double or_pair_f(double r2, double eps, double sigma, double rc, double c2) {
  if (r2 >= rc * rc) return 0.0;
  double s = r2 / (sigma * sigma);
  double s3 = s * s * s, s7 = s3 * s3 * s;
  return eps / (sigma * sigma) * ((24.0 * s3 - 48.0) / s7 + 8.0 * c2);
}

/* Min image of one component for |d| < 1.5 L (the fixed formula). */
static double min_image(double d, double L) {
  if (d > 0.5 * L) d -= L;
  else if (d < -0.5 * L) d += L;
  return d;
}

/* Min image for unwrapped coordinates (any |d|): the same formula repeated. */
static double min_image_any(double d, double L) {
  while (d > 0.5 * L) d -= L;
  while (d < -0.5 * L) d += L;
  return d;
}

/*
 * FCC lattice (benchmark initial condition, Sec. 4.5): M^3 cubic cells of side
 * a = (4/rho)^(1/3), four sites per cell at a*(0,0,0), a*(0,1/2,1/2),
 * a*(1/2,0,1/2), a*(1/2,1/2,0).  Particle id order: ix outermost, then iy, iz,
 * then the basis site.  Returns the box length L = M a.
 */
double or_fcc_lattice(int64_t M, double rho, double* x) {
  static const double basis[4][3] = {{0.0, 0.0, 0.0}, {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0}};
  double a = cbrt(4.0 / rho);
  int64_t p = 0;
  for (int64_t ix = 0; ix < M; ++ix)
    for (int64_t iy = 0; iy < M; ++iy)
      for (int64_t iz = 0; iz < M; ++iz)
        for (int b = 0; b < 4; ++b) {
          x[3 * p + 0] = a * ((double)ix + basis[b][0]);
          x[3 * p + 1] = a * ((double)iy + basis[b][1]);
          x[3 * p + 2] = a * ((double)iz + basis[b][2]);
          ++p;
        }
  return a * (double)M;
}

/*
 * SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) used as a counter-based
 * generator: draw number k of stream `seed` is mix(seed + (k+1) * golden).
 */
static uint64_t splitmix_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t or_splitmix_at(uint64_t seed, uint64_t k) { return splitmix_at(seed, k); }

/* Uniform in (0, 1]: the top 53 bits plus one, times 2^-53. */
static double uniform_at(uint64_t seed, uint64_t k) {
  return (double)((splitmix_at(seed, k) >> 11) + 1) * 0x1.0p-53;
}

/*
 * Raw Gaussian velocity components before momentum removal and scaling.
 * Particle p uses draws 4p..4p+3.  Box-Muller (1958): with u1 = draw 4p,
 * u2 = draw 4p+1, rad = sqrt(-2 ln u1): vx = rad cos(2 pi u2),
 * vy = rad sin(2 pi u2); with u3 = draw 4p+2, u4 = draw 4p+3:
 * vz = sqrt(-2 ln u3) cos(2 pi u4).
 */
void or_gaussian_raw(int64_t N, uint64_t seed, double* v) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int64_t p = 0; p < N; ++p) {
    double u1 = uniform_at(seed, 4 * (uint64_t)p + 0), u2 = uniform_at(seed, 4 * (uint64_t)p + 1);
    double u3 = uniform_at(seed, 4 * (uint64_t)p + 2), u4 = uniform_at(seed, 4 * (uint64_t)p + 3);
    double r12 = sqrt(-2.0 * log(u1)), r34 = sqrt(-2.0 * log(u3));
    v[3 * p + 0] = r12 * cos(two_pi * u2);
    v[3 * p + 1] = r12 * sin(two_pi * u2);
    v[3 * p + 2] = r34 * cos(two_pi * u4);
  }
}

/*
 * Initial velocities at temperature T: Gaussian components, total momentum
 * removed (subtract the mean), then scaled so that sum v^2 = 3 (N-1) T
 * (3(N-1) degrees of freedom once the momentum is fixed; m = kB = 1).
 */
void or_init_velocities(int64_t N, double T, uint64_t seed, double* v) {
  or_gaussian_raw(N, seed, v);
  double mean[3] = {0.0, 0.0, 0.0};
  for (int64_t p = 0; p < N; ++p)
    for (int k = 0; k < 3; ++k) mean[k] += v[3 * p + k];
  for (int k = 0; k < 3; ++k) mean[k] /= (double)N;
  double sumsq = 0.0;
  for (int64_t p = 0; p < N; ++p)
    for (int k = 0; k < 3; ++k) {
      v[3 * p + k] -= mean[k];
      sumsq += v[3 * p + k] * v[3 * p + k];
    }
  double scale = (N > 1 && sumsq > 0.0) ? sqrt(3.0 * (double)(N - 1) * T / sumsq) : 0.0;
  for (int64_t i = 0; i < 3 * N; ++i) v[i] *= scale;
}

/*
 * Forces, potential energy and virial by the plain O(N^2) cutoff sum.
 * F_i = sum_{j != i, r_ij < rc} f(r_ij) (q_j - q_i);
 * PE  = sum_{i<j} V(r_ij);  W = sum_{i<j} (q_i - q_j) . F_ij = -sum_{i<j} f r^2.
 * Each i sums over all j (Newton's third law is not used), so the result does
 * not depend on the thread count.  pe / vir may be NULL.
 */
void or_forces(int64_t N, const double* x, double L, double eps, double sigma, double rc, double c2,
               double c0, double* F, double* pe, double* vir) {
  double* pe_i = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
  double* w_i = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < N; ++i) {
    double fi[3] = {0.0, 0.0, 0.0}, e = 0.0, w = 0.0;
    for (int64_t j = 0; j < N; ++j) {
      if (j == i) continue;
      double d[3];
      for (int k = 0; k < 3; ++k) d[k] = min_image_any(x[3 * j + k] - x[3 * i + k], L);
      double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (r2 >= rc * rc) continue;
      double f = or_pair_f(r2, eps, sigma, rc, c2);
      for (int k = 0; k < 3; ++k) fi[k] += f * d[k];
      e += 0.5 * or_pair_v(r2, eps, sigma, rc, c2, c0);
      w += -0.5 * f * r2;
    }
    for (int k = 0; k < 3; ++k) F[3 * i + k] = fi[k];
    pe_i[i] = e;
    w_i[i] = w;
  }
  double e = 0.0, w = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    e += pe_i[i];
    w += w_i[i];
  }
  if (pe) *pe = e;
  if (vir) *vir = w;
  free(pe_i);
  free(w_i);
}

/* Forces on a sample of particles idx[0..ns) only (same sum as or_forces). */
void or_forces_sample(int64_t N, const double* x, double L, double eps, double sigma, double rc, double c2,
                      const int64_t* idx, int64_t ns, double* F) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t s = 0; s < ns; ++s) {
    int64_t i = idx[s];
    double fi[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < N; ++j) {
      if (j == i) continue;
      double d[3];
      for (int k = 0; k < 3; ++k) d[k] = min_image_any(x[3 * j + k] - x[3 * i + k], L);
      double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (r2 >= rc * rc) continue;
      double f = or_pair_f(r2, eps, sigma, rc, c2);
      for (int k = 0; k < 3; ++k) fi[k] += f * d[k];
    }
    for (int k = 0; k < 3; ++k) F[3 * s + k] = fi[k];
  }
}

double or_kinetic(int64_t N, const double* v) {
  double s = 0.0;
  for (int64_t i = 0; i < 3 * N; ++i) s += v[i] * v[i];
  return 0.5 * s;
}

/*
 * Velocity-Verlet ("second-order symplectic", Sec. 4.5), m = 1:
 *   v <- v + (dt/2) F(x);  x <- x + dt v;  v <- v + (dt/2) F(x).
 * F must hold F(x) on entry and holds F(x) on exit.  Positions are not
 * wrapped (the min image handles the periodic box), so x stays unwrapped.
 * If pe_t / ke_t are given they receive PE and KE after each step.
 */
void or_vv_run(int64_t N, double* x, double* v, double* F, double L, double eps, double sigma, double rc,
               double c2, double c0, double dt, int64_t nsteps, double* pe_t, double* ke_t, double* vir_t) {
  const double h = 0.5 * dt;
  for (int64_t n = 0; n < nsteps; ++n) {
    for (int64_t i = 0; i < 3 * N; ++i) v[i] += h * F[i];
    for (int64_t i = 0; i < 3 * N; ++i) x[i] += dt * v[i];
    double pe, vir;
    or_forces(N, x, L, eps, sigma, rc, c2, c0, F, &pe, &vir);
    for (int64_t i = 0; i < 3 * N; ++i) v[i] += h * F[i];
    if (pe_t) pe_t[n] = pe;
    if (ke_t) ke_t[n] = or_kinetic(N, v);
    if (vir_t) vir_t[n] = vir;
  }
}

/*
 * Brute-force pair set within the search length (Alg. 1's "interact"
 * test with r < rs, strict): every (i, j), i < j, with r_ij^2 < rs^2, where
 * r^2 = dx*dx + dy*dy + dz*dz evaluated left to right without FMA, on the
 * fixed min-image differences of wrapped positions.  Pairs are written in
 * lexicographic order as (i, j) into ij[2*k], ij[2*k+1] while k < cap.
 * Returns the total count (which may exceed cap).
 */
int64_t or_pairs_within(int64_t N, const double* x, double L, double rs, int64_t* ij, int64_t cap) {
  int64_t count = 0;
  const double rs2 = rs * rs;
  for (int64_t i = 0; i < N; ++i)
    for (int64_t j = i + 1; j < N; ++j) {
      double dx = min_image(x[3 * j + 0] - x[3 * i + 0], L);
      double dy = min_image(x[3 * j + 1] - x[3 * i + 1], L);
      double dz = min_image(x[3 * j + 2] - x[3 * i + 2], L);
      double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 < rs2) {
        if (count < cap) {
          ij[2 * count] = i;
          ij[2 * count + 1] = j;
        }
        ++count;
      }
    }
  return count;
}

/* Count of pairs within rs per particle (full count, both directions). */
void or_neighbor_counts(int64_t N, const double* x, double L, double rs, int64_t* cnt) {
  const double rs2 = rs * rs;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < N; ++i) {
    int64_t c = 0;
    for (int64_t j = 0; j < N; ++j) {
      if (j == i) continue;
      double dx = min_image(x[3 * j + 0] - x[3 * i + 0], L);
      double dy = min_image(x[3 * j + 1] - x[3 * i + 1], L);
      double dz = min_image(x[3 * j + 2] - x[3 * i + 2], L);
      double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 < rs2) ++c;
    }
    cnt[i] = c;
  }
}

/* ---------------------------------------------------------------------------
 * Derivatives for the adjoint (differentiation form).  The paper has no
 * adjoint; these are the plain derivatives of the Eq. 2 pair energy written as
 * a function of s = r^2 (not divided by sigma^2 here):
 *   u(s)   = 4 eps [ sigma^12 s^-6 - sigma^6 s^-3 + c2 s / sigma^2 + c0 ]
 *   u'(s)  = 4 eps [ -6 sigma^12 s^-7 + 3 sigma^6 s^-4 + c2 / sigma^2 ]
 *   u''(s) = 4 eps [ 42 sigma^12 s^-8 - 12 sigma^6 s^-5 ]
 * With d_ij = q_i - q_j, U = sum_{i<j} u(s_ij):
 *   dU/dq_i = sum_j 2 u'(s) d_ij            (so F_i = -sum_j 2 u'(s) d_ij)
 *   (H w)_i = sum_j [ 2 u'(s) (w_i - w_j) + 4 u''(s) d_ij (d_ij . (w_i - w_j)) ]
 * Sigma derivatives hold rc/sigma fixed, so c2 and c0 are constants; the
 * boundary terms of the moving cutoff vanish because V(rc) = V'(rc) = 0.
 * ------------------------------------------------------------------------- */
static void pair_u_derivs(double s, double eps, double sigma, double c2, double c0, double* u, double* u1,
                          double* u2, double* du_de, double* du_ds, double* du1_de, double* du1_ds) {
  double sg2 = sigma * sigma, sg6 = sg2 * sg2 * sg2, sg12 = sg6 * sg6;
  double is = 1.0 / s, is3 = is * is * is, is6 = is3 * is3;
  double v = 4.0 * eps * (sg12 * is6 - sg6 * is3 + c2 * s / sg2 + c0);
  double d1 = 4.0 * eps * (-6.0 * sg12 * is6 * is + 3.0 * sg6 * is3 * is + c2 / sg2);
  double d2 = 4.0 * eps * (42.0 * sg12 * is6 * is * is - 12.0 * sg6 * is3 * is * is);
  if (u) *u = v;
  if (u1) *u1 = d1;
  if (u2) *u2 = d2;
  if (du_de) *du_de = v / eps;
  if (du1_de) *du1_de = d1 / eps;
  if (du_ds) *du_ds = 4.0 * eps * (12.0 * sg12 / sigma * is6 - 6.0 * sg6 / sigma * is3 - 2.0 * c2 * s / (sg2 * sigma));
  if (du1_ds)
    *du1_ds = 4.0 * eps * (-72.0 * sg12 / sigma * is6 * is + 18.0 * sg6 / sigma * is3 * is - 2.0 * c2 / (sg2 * sigma));
}

/* Hessian-vector product H(x) w of the potential energy (pairs with r < rc). */
void or_hvp(int64_t N, const double* x, double L, double eps, double sigma, double rc, double c2, double c0,
            const double* w, double* Hw) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < N; ++i) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < N; ++j) {
      if (j == i) continue;
      double d[3];
      for (int k = 0; k < 3; ++k) d[k] = min_image_any(x[3 * i + k] - x[3 * j + k], L);
      double s = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (s >= rc * rc) continue;
      double u1, u2;
      pair_u_derivs(s, eps, sigma, c2, c0, NULL, &u1, &u2, NULL, NULL, NULL, NULL);
      double dw[3] = {w[3 * i] - w[3 * j], w[3 * i + 1] - w[3 * j + 1], w[3 * i + 2] - w[3 * j + 2]};
      double ddw = d[0] * dw[0] + d[1] * dw[1] + d[2] * dw[2];
      for (int k = 0; k < 3; ++k) acc[k] += 2.0 * u1 * dw[k] + 4.0 * u2 * d[k] * ddw;
    }
    for (int k = 0; k < 3; ++k) Hw[3 * i + k] = acc[k];
  }
}

/*
 * Dense Hessian of the potential energy, H[(3i+a)*3N + (3j+b)] = d2U/dq_ia dq_jb,
 * assembled pair by pair from the second derivative of u(|q_i - q_j|^2):
 *   block (i,i) += 2u' I + 4u'' d d^T,  block (i,j) -= 2u' I + 4u'' d d^T.
 * For small N only (the matrix has 9 N^2 entries).
 */
void or_hessian(int64_t N, const double* x, double L, double eps, double sigma, double rc, double c2, double c0,
                double* H) {
  int64_t n3 = 3 * N;
  memset(H, 0, sizeof(double) * (size_t)(n3 * n3));
  for (int64_t i = 0; i < N; ++i)
    for (int64_t j = 0; j < N; ++j) {
      if (j == i) continue;
      double d[3];
      for (int k = 0; k < 3; ++k) d[k] = min_image_any(x[3 * i + k] - x[3 * j + k], L);
      double s = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (s >= rc * rc) continue;
      double u1, u2;
      pair_u_derivs(s, eps, sigma, c2, c0, NULL, &u1, &u2, NULL, NULL, NULL, NULL);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double blk = (a == b ? 2.0 * u1 : 0.0) + 4.0 * u2 * d[a] * d[b];
          H[(3 * i + a) * n3 + (3 * i + b)] += blk;
          H[(3 * i + a) * n3 + (3 * j + b)] -= blk;
        }
    }
}

/*
 * Parameter derivatives at configuration x:
 *   dpe[0] = dPE/deps, dpe[1] = dPE/dsigma
 *   vjp[0] = lam . dF/deps, vjp[1] = lam . dF/dsigma  (lam may be NULL)
 * with F_i = -sum_j 2 u'(s_ij) d_ij, so lam . dF/dtheta =
 *   -sum_{i<j} 2 (du'/dtheta)(s_ij) d_ij . (lam_i - lam_j).
 */
void or_param_derivs(int64_t N, const double* x, double L, double eps, double sigma, double rc, double c2, double c0,
                     const double* lam, double* dpe, double* vjp) {
  double* acc = (double*)calloc((size_t)(N > 0 ? N : 1) * 4, sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < N; ++i) {
    double a_de = 0.0, a_ds = 0.0, l_de = 0.0, l_ds = 0.0;
    for (int64_t j = 0; j < N; ++j) {
      if (j == i) continue;
      double d[3];
      for (int k = 0; k < 3; ++k) d[k] = min_image_any(x[3 * i + k] - x[3 * j + k], L);
      double s = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (s >= rc * rc) continue;
      double du_de, du_ds, du1_de, du1_ds;
      pair_u_derivs(s, eps, sigma, c2, c0, NULL, NULL, NULL, &du_de, &du_ds, &du1_de, &du1_ds);
      a_de += 0.5 * du_de;
      a_ds += 0.5 * du_ds;
      if (lam) {
        double dl = d[0] * (lam[3 * i] - lam[3 * j]) + d[1] * (lam[3 * i + 1] - lam[3 * j + 1]) +
                    d[2] * (lam[3 * i + 2] - lam[3 * j + 2]);
        l_de += -0.5 * 2.0 * du1_de * dl;
        l_ds += -0.5 * 2.0 * du1_ds * dl;
      }
    }
    acc[4 * i + 0] = a_de;
    acc[4 * i + 1] = a_ds;
    acc[4 * i + 2] = l_de;
    acc[4 * i + 3] = l_ds;
  }
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    s0 += acc[4 * i];
    s1 += acc[4 * i + 1];
    s2 += acc[4 * i + 2];
    s3 += acc[4 * i + 3];
  }
  if (dpe) {
    dpe[0] = s0;
    dpe[1] = s1;
  }
  if (vjp) {
    vjp[0] = s2;
    vjp[1] = s3;
  }
  free(acc);
}

/*
 * Loss of the differentiable trajectory and its exact FP64 gradient.
 *   loss = (1/n_pe) sum_{t = nsteps-n_pe+1}^{nsteps} PE(x_t) / N
 *        + (1/N) sum_i |x_i(nsteps) - x_i(0)|^2        (unwrapped positions)
 * Forward: nsteps of velocity-Verlet from (x0, v0), all states kept.
 * Reverse (h = dt/2), for one step  v' = v + h F(x), x+ = x + dt v',
 * v+ = v' + h F(x+), given adjoints (lx+, lv+):
 *   lv'  = lv+ ;  lx+ <- lx+ - h H(x+) lv+ ;  ltheta += h (dF/dtheta)(x+)^T lv+
 *   lv'  += dt lx+ ;  lx = lx+ ;  lx <- lx - h H(x) lv' ;  lv = lv'
 *   ltheta += h (dF/dtheta)(x)^T lv'
 * Direct terms: dloss/dx_t = -F(x_t) / (n_pe N) on the averaged steps,
 * +2 (x_n - x_0)/N at t = nsteps and -2 (x_n - x_0)/N at t = 0;
 * dloss/dtheta gets (1/(n_pe N)) dPE/dtheta at every averaged step.
 * Outputs: *loss, gx0[3N], gv0[3N] (may be NULL), gtheta[2] = (d/deps, d/dsigma).
 */
void or_traj_loss_grad(int64_t N, const double* x0, const double* v0, double L, double eps, double sigma, double rc,
                       double c2, double c0, double dt, int64_t nsteps, int64_t n_pe, double* loss, double* gx0,
                       double* gv0, double* gtheta) {
  const double h = 0.5 * dt;
  size_t n3 = (size_t)(3 * N);
  double* xs = (double*)malloc(sizeof(double) * n3 * (size_t)(nsteps + 1));
  double* vs = (double*)malloc(sizeof(double) * n3 * (size_t)(nsteps + 1));
  double* F = (double*)malloc(sizeof(double) * n3);
  double* tmp = (double*)malloc(sizeof(double) * n3);
  double* lx = (double*)malloc(sizeof(double) * n3);
  double* lv = (double*)malloc(sizeof(double) * n3);
  memcpy(xs, x0, sizeof(double) * n3);
  memcpy(vs, v0, sizeof(double) * n3);
  double pe = 0.0, acc_pe = 0.0;
  or_forces(N, xs, L, eps, sigma, rc, c2, c0, F, &pe, NULL);
  for (int64_t n = 0; n < nsteps; ++n) {
    double* xc = xs + n3 * (size_t)n;
    double* vc = vs + n3 * (size_t)n;
    double* xn = xc + n3;
    double* vn = vc + n3;
    for (size_t i = 0; i < n3; ++i) vn[i] = vc[i] + h * F[i];
    for (size_t i = 0; i < n3; ++i) xn[i] = xc[i] + dt * vn[i];
    or_forces(N, xn, L, eps, sigma, rc, c2, c0, F, &pe, NULL);
    for (size_t i = 0; i < n3; ++i) vn[i] += h * F[i];
    if (n + 1 > nsteps - n_pe) acc_pe += pe;
  }
  const double* xN = xs + n3 * (size_t)nsteps;
  double msd = 0.0;
  for (size_t i = 0; i < n3; ++i) msd += (xN[i] - x0[i]) * (xN[i] - x0[i]);
  const double wpe = 1.0 / ((double)n_pe * (double)N);
  *loss = acc_pe * wpe + msd / (double)N;

  double gth[2] = {0.0, 0.0};
  /* direct terms at t = nsteps */
  or_forces(N, xN, L, eps, sigma, rc, c2, c0, F, NULL, NULL);
  for (size_t i = 0; i < n3; ++i) {
    lx[i] = 2.0 * (xN[i] - x0[i]) / (double)N;
    lv[i] = 0.0;
  }
  if (n_pe > 0) {
    double dpe[2];
    for (size_t i = 0; i < n3; ++i) lx[i] += -F[i] * wpe;
    or_param_derivs(N, xN, L, eps, sigma, rc, c2, c0, NULL, dpe, NULL);
    gth[0] += dpe[0] * wpe;
    gth[1] += dpe[1] * wpe;
  }
  for (int64_t n = nsteps - 1; n >= 0; --n) {
    const double* xc = xs + n3 * (size_t)n;
    const double* xp = xc + n3;
    double vj[2];
    /* v+ = v' + h F(x+) */
    or_hvp(N, xp, L, eps, sigma, rc, c2, c0, lv, tmp);
    for (size_t i = 0; i < n3; ++i) lx[i] -= h * tmp[i];
    or_param_derivs(N, xp, L, eps, sigma, rc, c2, c0, lv, NULL, vj);
    gth[0] += h * vj[0];
    gth[1] += h * vj[1];
    /* x+ = x + dt v' */
    for (size_t i = 0; i < n3; ++i) lv[i] += dt * lx[i];
    /* v' = v + h F(x) */
    or_hvp(N, xc, L, eps, sigma, rc, c2, c0, lv, tmp);
    for (size_t i = 0; i < n3; ++i) lx[i] -= h * tmp[i];
    or_param_derivs(N, xc, L, eps, sigma, rc, c2, c0, lv, NULL, vj);
    gth[0] += h * vj[0];
    gth[1] += h * vj[1];
    /* direct terms at state n */
    if (n > nsteps - n_pe) {
      double dpe[2];
      or_forces(N, xc, L, eps, sigma, rc, c2, c0, F, NULL, NULL);
      for (size_t i = 0; i < n3; ++i) lx[i] += -F[i] * wpe;
      or_param_derivs(N, xc, L, eps, sigma, rc, c2, c0, NULL, dpe, NULL);
      gth[0] += dpe[0] * wpe;
      gth[1] += dpe[1] * wpe;
    }
    if (n == 0)
      for (size_t i = 0; i < n3; ++i) lx[i] += -2.0 * (xN[i] - x0[i]) / (double)N;
  }
  memcpy(gx0, lx, sizeof(double) * n3);
  if (gv0) memcpy(gv0, lv, sizeof(double) * n3);
  gtheta[0] = gth[0];
  gtheta[1] = gth[1];
  free(xs);
  free(vs);
  free(F);
  free(tmp);
  free(lx);
  free(lv);
}

/* Loss alone (forward only), for finite differences of the oracle itself. */
double or_traj_loss(int64_t N, const double* x0, const double* v0, double L, double eps, double sigma, double rc,
                    double c2, double c0, double dt, int64_t nsteps, int64_t n_pe) {
  const double h = 0.5 * dt;
  size_t n3 = (size_t)(3 * N);
  double* x = (double*)malloc(sizeof(double) * n3);
  double* v = (double*)malloc(sizeof(double) * n3);
  double* F = (double*)malloc(sizeof(double) * n3);
  memcpy(x, x0, sizeof(double) * n3);
  memcpy(v, v0, sizeof(double) * n3);
  double pe, acc_pe = 0.0;
  or_forces(N, x, L, eps, sigma, rc, c2, c0, F, &pe, NULL);
  for (int64_t n = 0; n < nsteps; ++n) {
    for (size_t i = 0; i < n3; ++i) v[i] += h * F[i];
    for (size_t i = 0; i < n3; ++i) x[i] += dt * v[i];
    or_forces(N, x, L, eps, sigma, rc, c2, c0, F, &pe, NULL);
    for (size_t i = 0; i < n3; ++i) v[i] += h * F[i];
    if (n + 1 > nsteps - n_pe) acc_pe += pe;
  }
  double msd = 0.0;
  for (size_t i = 0; i < n3; ++i) msd += (x[i] - x0[i]) * (x[i] - x0[i]);
  free(x);
  free(v);
  free(F);
  return acc_pe / ((double)n_pe * (double)N) + msd / (double)N;
}
