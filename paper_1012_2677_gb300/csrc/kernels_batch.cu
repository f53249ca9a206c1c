// Batched replicas: the per-replica pieces of the rebuild and the reductions.  Particles of
// replica r occupy [base_r, base_r + count_r) of every particle array and never leave it (the
// cell sort permutes inside a replica's cells); rep_of[i] names the replica of particle i.
// Kernels that belong to the rebuild take a device flag and return at once when it is zero, so
// that a captured graph of K steps can carry the rebuild and run it only when the displacement
// rule asks for it.
#include "common.cuh"

namespace ljmd {

static int grid_of(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  return (int)(b < 1048576 ? b : 1048576);
}

// Fold into the replica's box (img counts the folds) and label by the replica's cell grid;
// global cell = cell_base + (cx n + cy) n + cz.  Same arithmetic as the single-system labelling.
__global__ void k_wrap_label_batch(double* __restrict__ x, int32_t* __restrict__ img, int64_t N,
                                   const int32_t* __restrict__ rep_of, const ReplicaGeo* __restrict__ reps,
                                   double offset, uint32_t* __restrict__ cell_of, uint32_t* __restrict__ count,
                                   int32_t* __restrict__ status, const int* __restrict__ pred) {
  if (pred && !*pred) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const ReplicaGeo& rg = reps[rep_of[i]];
    const Geom& g = rg.g;
    int c[3];
    bool bad = false;
    for (int k = 0; k < 3; ++k) {
      double xs = x[k * N + i];
      if (!finite_d(xs)) bad = true;
      if (cmp_ge_d(xs, offset + g.L)) {
        xs -= g.L;
        img[k * N + i] += 1;
        x[k * N + i] = xs;
      } else if (!cmp_ge_d(xs, offset)) {
        xs += g.L;
        img[k * N + i] -= 1;
        x[k * N + i] = xs;
      }
      int ck = floor_to_int((xs - offset) * g.inv_h);
      ck = ck < 0 ? 0 : (ck >= g.n ? g.n - 1 : ck);
      c[k] = ck;
    }
    if (bad) {
      atomicOr(status, LJ_ST_NONFINITE);
      c[0] = c[1] = c[2] = 0;
    }
    const uint32_t cell =
        (uint32_t)rg.cell_base + ((uint32_t)c[0] * (uint32_t)g.n + (uint32_t)c[1]) * (uint32_t)g.n + (uint32_t)c[2];
    cell_of[i] = cell;
    atomicAdd(&count[cell], 1u);
  }
}
void launch_wrap_label_batch(double* x, int32_t* img, int64_t N, const int32_t* rep_of, const ReplicaGeo* reps,
                             double offset, uint32_t* cell_of, uint32_t* cell_count, int32_t* status,
                             const int* pred, cudaStream_t s) {
  k_wrap_label_batch<<<grid_of(N), 256, 0, s>>>(x, img, N, rep_of, reps, offset, cell_of, cell_count, status, pred);
}

// Displacement rule on the device: flag = (largest squared displacement since the build >
// limit^2); every raised flag is counted.
__global__ void k_rebuild_flag(const uint32_t* __restrict__ dmax_bits, float limit2, int* __restrict__ flag,
                               long long* __restrict__ rebuilds) {
  const int f = __uint_as_float(*dmax_bits) > limit2 ? 1 : 0;
  *flag = f;
  if (f) *rebuilds += 1;
}
void launch_rebuild_flag(const uint32_t* dmax_bits, float limit2, int* flag, long long* rebuilds, cudaStream_t s) {
  k_rebuild_flag<<<1, 1, 0, s>>>(dmax_bits, limit2, flag, rebuilds);
}

// Predicated copy of `bytes` (a multiple of 4) from in to out: 16-byte words while both
// addresses are 16-byte aligned (the device allocations are), then the 4-byte tail.
__global__ void k_copy_words(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n,
                             const int* __restrict__ pred) {
  if (pred && !*pred) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t n16 = 0;
  if ((((uintptr_t)in | (uintptr_t)out) & 15u) == 0) {
    n16 = n / 4;
    const uint4* __restrict__ a = (const uint4*)in;
    uint4* __restrict__ b = (uint4*)out;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n16; i += stride) b[i] = a[i];
  }
  for (int64_t i = 4 * n16 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) out[i] = in[i];
}
void launch_copy_words(const void* in, void* out, int64_t bytes, const int* pred, cudaStream_t s) {
  const int64_t n = bytes / 4;
  k_copy_words<<<grid_of((n + 3) / 4), 256, 0, s>>>((const uint32_t*)in, (uint32_t*)out, n, pred);
}

// Predicated zero fill of `bytes` (a multiple of 4).
__global__ void k_zero_words(uint32_t* __restrict__ out, int64_t n, const int* __restrict__ pred) {
  if (pred && !*pred) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = 0u;
}
void launch_zero_words(void* out, int64_t bytes, const int* pred, cudaStream_t s) {
  const int64_t n = bytes / 4;
  k_zero_words<<<grid_of(n), 256, 0, s>>>((uint32_t*)out, n, pred);
}

// Kinetic energy per replica, 1/2 sum v^2 over its particles: blockIdx.y = replica, the blocks
// along x stride over its particles; one FP64 atomic per block.
__global__ void k_replica_ke(const double* __restrict__ v, int64_t N, const ReplicaGeo* __restrict__ reps,
                             double* __restrict__ ke_rep) {
  __shared__ double sh[32];
  const ReplicaGeo& rg = reps[blockIdx.y];
  double acc = 0.0;
  for (int64_t i = rg.base + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rg.base + rg.count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double a = v[i], b = v[N + i], c = v[2 * N + i];
    acc += 0.5 * (a * a + b * b + c * c);
  }
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0 && t != 0.0) atomicAdd(&ke_rep[blockIdx.y], t);
}
void launch_replica_ke(const double* v, int64_t N, const ReplicaGeo* reps, int R, double* ke_rep, cudaStream_t s) {
  dim3 grid(8, (unsigned)R);
  k_replica_ke<<<grid, 256, 0, s>>>(v, N, reps, ke_rep);
}

// Caller-order AoS into the SoA state of a batch (id = i): positions folded into their replica's
// box (img counts the folds) and stored as offset + x; velocities copied (zero if vin is null).
__global__ void k_load_batch(const double* __restrict__ xin, const double* __restrict__ vin, double* __restrict__ x,
                             double* __restrict__ v, int32_t* __restrict__ id, int32_t* __restrict__ img, int64_t N,
                             const int32_t* __restrict__ rep_of, const ReplicaGeo* __restrict__ reps, double offset) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    const double L = reps[rep_of[p]].g.L;
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
void launch_load_batch(const double* xin, const double* vin, double* x, double* v, int32_t* id, int32_t* img,
                       int64_t N, const int32_t* rep_of, const ReplicaGeo* reps, double offset, cudaStream_t s) {
  k_load_batch<<<grid_of(N), 256, 0, s>>>(xin, vin, x, v, id, img, N, rep_of, reps, offset);
}

}  // namespace ljmd
