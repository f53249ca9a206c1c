// Initial state (FCC lattice + Gaussian velocities) and the fixed-order reductions.
#include <math.h>

#include "common.cuh"

namespace ljmd {

int red_blocks(int64_t n) {
  int64_t b = (n + kRedThreads - 1) / kRedThreads;
  if (b < 1) b = 1;
  return (int)(b < kMaxRedBlocks ? b : kMaxRedBlocks);
}

// ---------------------------------------------------------------------------------------------
// Final reduction: out[q] = sum over blocks of partials[b * nq + q], q < nq <= 4, one block,
// fixed order (thread t sums blocks t, t + 1024, ...; then the block tree).
__global__ void k_final_reduce(const double* __restrict__ part, int nb, int nq, double* __restrict__ out) {
  __shared__ double sh[32];
  for (int q = 0; q < nq; ++q) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[(size_t)b * nq + q];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) out[q] = s;
    __syncthreads();
  }
}

void launch_final_reduce(const double* partials, int nblocks, int nq, double* out, cudaStream_t s) {
  k_final_reduce<<<1, 1024, 0, s>>>(partials, nblocks, nq, out);
}

// energies[0..3] = (pe, ke, virial, step).  pe/vir from the force partials (scaled by
// pe_scale: 1/2 for a full list, where every pair is visited twice), ke from the
// integrator partials.  Appends (step, pe, ke, vir) to the log if there is room.
__global__ void k_energy_finalize(const double* __restrict__ pv, int nbf, const double* __restrict__ kp, int nbi,
                                  double pe_scale, double* __restrict__ energies, double* __restrict__ log,
                                  int64_t cap, int64_t* __restrict__ count, double step,
                                  const int* __restrict__ skip) {
  if (skip && *skip) return;  // a device-decided run stopped before this step
  energy_record_block(pv, nbf, kp, nbi, pe_scale, energies, log, cap, count, step);
}

void launch_energy_finalize(const double* pe_vir_part, int nb_force, const double* ke_part, int nb_int,
                            double pe_scale, double* energies, double* log, int64_t log_cap, int64_t* log_count,
                            double step, cudaStream_t s, const int* skip) {
  k_energy_finalize<<<1, 1024, 0, s>>>(pe_vir_part, nb_force, ke_part, nb_int, pe_scale, energies, log, log_cap,
                                        log_count, step, skip);
}

// ---------------------------------------------------------------------------------------------
// FCC lattice of the benchmark (Sec. 4.5): id p = ((ix M + iy) M + iz) 4 + b at
// a ((ix, iy, iz) + basis_b), stored as offset + coordinate (SoA x[k * N + p]).
__global__ void k_fcc(double* __restrict__ x, int64_t M, double a, double offset) {
  const int64_t N = 4 * M * M * M;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(p & 3);
    const int64_t cell = p >> 2;
    const int64_t iz = cell % M, iy = (cell / M) % M, ix = cell / (M * M);
    // basis (0,0,0), (0,1/2,1/2), (1/2,0,1/2), (1/2,1/2,0)
    const double bx = (b == 2 || b == 3) ? 0.5 : 0.0;
    const double by = (b == 1 || b == 3) ? 0.5 : 0.0;
    const double bz = (b == 1 || b == 2) ? 0.5 : 0.0;
    x[p] = offset + a * ((double)ix + bx);
    x[N + p] = offset + a * ((double)iy + by);
    x[2 * N + p] = offset + a * ((double)iz + bz);
  }
}

void launch_fcc(double* x, int64_t M, double a, double offset, cudaStream_t s) {
  const int64_t N = 4 * M * M * M;
  int blocks = (int)((N + 255) / 256);
  if (blocks > 65535) blocks = 65535;
  k_fcc<<<blocks, 256, 0, s>>>(x, M, a, offset);
}

// Counter-based SplitMix64: draw k of stream `seed` is mix(seed + (k + 1) * golden)
// (Steele, Lea and Flood 2014).  Uniform in (0, 1] from the top 53 bits plus one.
__device__ __forceinline__ uint64_t sm64_draw(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double sm64_uniform(uint64_t seed, uint64_t k) {
  return (double)((sm64_draw(seed, k) >> 11) + 1) * 0x1.0p-53;
}

// Box-Muller on draws 4p..4p+3: vx, vy from (u1, u2), vz from (u3, u4).
__global__ void k_gaussian(double* __restrict__ v, int64_t N, uint64_t seed) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = 4 * (uint64_t)p;
    const double u1 = sm64_uniform(seed, k), u2 = sm64_uniform(seed, k + 1);
    const double u3 = sm64_uniform(seed, k + 2), u4 = sm64_uniform(seed, k + 3);
    const double r12 = sqrt(-2.0 * log(u1)), r34 = sqrt(-2.0 * log(u3));
    double sn, cs;
    sincos(two_pi * u2, &sn, &cs);
    v[p] = r12 * cs;
    v[N + p] = r12 * sn;
    v[2 * N + p] = r34 * cos(two_pi * u4);
  }
}

void launch_gaussian(double* v, int64_t N, uint64_t seed, cudaStream_t s) {
  int blocks = (int)((N + 255) / 256);
  if (blocks > 65535) blocks = 65535;
  k_gaussian<<<blocks, 256, 0, s>>>(v, N, seed);
}

// Per-block partial sums of the three velocity components.
__global__ void k_sums3(const double* __restrict__ v, int64_t N, double* __restrict__ part) {
  __shared__ double sh[32];
  double s[3] = {0.0, 0.0, 0.0};
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x)
    for (int k = 0; k < 3; ++k) s[k] += v[k * N + p];
  for (int k = 0; k < 3; ++k) {
    double t = block_sum(s[k], sh);
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * 3 + k] = t;
    __syncthreads();
  }
}

void launch_sums3(const double* v, int64_t N, double* partials, int nb, cudaStream_t s) {
  k_sums3<<<nb, kRedThreads, 0, s>>>(v, N, partials);
}

// Per-block partial sums of |v - mean|^2, mean = sums / N.
__global__ void k_sumsq_centered(const double* __restrict__ v, int64_t N, const double* __restrict__ sums,
                                 double* __restrict__ part) {
  __shared__ double sh[32];
  const double m0 = sums[0] / (double)N, m1 = sums[1] / (double)N, m2 = sums[2] / (double)N;
  double s = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    const double a = v[p] - m0, b = v[N + p] - m1, c = v[2 * N + p] - m2;
    s += a * a + b * b + c * c;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

void launch_sumsq_centered(const double* v, int64_t N, const double* sums, double* partials, int nb,
                           cudaStream_t s) {
  k_sumsq_centered<<<nb, kRedThreads, 0, s>>>(v, N, sums, partials);
}

// v <- (v - mean) * sqrt(3 (N - 1) T / sum |v - mean|^2): zero momentum, kinetic temperature T.
__global__ void k_center_scale(double* __restrict__ v, int64_t N, const double* __restrict__ sums,
                               const double* __restrict__ sumsq, double T) {
  const double m0 = sums[0] / (double)N, m1 = sums[1] / (double)N, m2 = sums[2] / (double)N;
  const double ss = sumsq[0];
  const double scale = (N > 1 && ss > 0.0) ? sqrt(3.0 * (double)(N - 1) * T / ss) : 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    v[p] = (v[p] - m0) * scale;
    v[N + p] = (v[N + p] - m1) * scale;
    v[2 * N + p] = (v[2 * N + p] - m2) * scale;
  }
}

void launch_center_scale(double* v, int64_t N, const double* sums, const double* sumsq, double T, cudaStream_t s) {
  int blocks = (int)((N + 255) / 256);
  if (blocks > 65535) blocks = 65535;
  k_center_scale<<<blocks, 256, 0, s>>>(v, N, sums, sumsq, T);
}

}  // namespace ljmd
