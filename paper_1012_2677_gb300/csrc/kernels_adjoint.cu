// Element-wise kernels of the reverse-time (adjoint) pass through velocity-Verlet: moving adjoint
// vectors between the caller's id order and the library's cell-sorted order, the unwrapped
// trajectory state, and the vector updates of the recurrences.  The pair work (Hessian-vector
// product, forces and parameter derivatives) is the adjoint tile kernel of kernels_tile.cu.
#include "common.cuh"

namespace ljmd {

static int grid_of(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  return (int)(b < 65535 ? b : 65535);
}

// w_sorted[s] = (w[3 id[s]], w[3 id[s] + 1], w[3 id[s] + 2]) (or zero when w is null), and its FP32
// copy (rounded to nearest) for the mixed form's pair loop.
__global__ void k_to_sorted(const double* __restrict__ w, const int32_t* __restrict__ id, int64_t N,
                            dvec4* __restrict__ out, float4* __restrict__ out32) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
    dvec4 v = make_dvec4(0.0, 0.0, 0.0, 0.0);
    if (w) {
      const int64_t p = id[s];
      v = make_dvec4(w[3 * p], w[3 * p + 1], w[3 * p + 2], 0.0);
    }
    out[s] = v;
    out32[s] = make_float4((float)v.x, (float)v.y, (float)v.z, 0.0f);
  }
}
void launch_to_sorted(const double* w_id, const int32_t* id, int64_t N, dvec4* out, float4* out32, cudaStream_t s) {
  k_to_sorted<<<grid_of(N), 256, 0, s>>>(w_id, id, N, out, out32);
}

// Unwrapped positions in id order: out[3 id[s] + k] = x[k N + s] - offset + img[k N + s] L.  Inside a
// device-decided run (ctl non-null, after the drift of its step k) nothing is written if the run
// stopped at an earlier step (the drift of step k did not happen).
__global__ void k_unwrapped(const double* __restrict__ x, const int32_t* __restrict__ img,
                            const int32_t* __restrict__ id, int64_t N, double offset, double L,
                            double* __restrict__ out, const StepCtl* __restrict__ ctl, int k_step) {
  if (ctl && ctl->stop && ctl->stop_at < k_step) return;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = id[s];
#pragma unroll
    for (int k = 0; k < 3; ++k) out[3 * p + k] = (x[k * N + s] - offset) + (double)img[k * N + s] * L;
  }
}
void launch_unwrapped(const double* x, const int32_t* img, const int32_t* id, int64_t N, double offset, double L,
                      double* out, cudaStream_t s, const StepCtl* ctl, int k_step) {
  k_unwrapped<<<grid_of(N), 256, 0, s>>>(x, img, id, N, offset, L, out, ctl, k_step);
}

// The inverse of k_unwrapped for the current sorted order and image counts: x[k N + s] =
// offset + u[3 id[s] + k] - img[k N + s] L, so that positions given unwrapped in id order are
// stored without re-sorting the particles (the list built for this order stays usable while the
// displacement rule holds).
__global__ void k_load_unwrapped(const double* __restrict__ u, const int32_t* __restrict__ img,
                                 const int32_t* __restrict__ id, int64_t N, double offset, double L,
                                 double* __restrict__ x) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = id[s];
#pragma unroll
    for (int k = 0; k < 3; ++k) x[k * N + s] = offset + (u[3 * p + k] - (double)img[k * N + s] * L);
  }
}
void launch_load_unwrapped(const double* u, const int32_t* img, const int32_t* id, int64_t N, double offset, double L,
                           double* x, cudaStream_t s) {
  k_load_unwrapped<<<grid_of(N), 256, 0, s>>>(u, img, id, N, offset, L, x);
}

// Parameter-gradient accumulation on the device: gth[0] += a0 q[0] + a4 q[4], gth[1] += a1 q[1] +
// a3 q[3], with q the five reduced sums of an adjoint pass (one thread).
__global__ void k_accum_q(const double* __restrict__ q, double a0, double a1, double a3, double a4,
                          double* __restrict__ gth) {
  gth[0] += a0 * q[0] + a4 * q[4];
  gth[1] += a1 * q[1] + a3 * q[3];
}
void launch_accum_q(const double* q, double a0, double a1, double a3, double a4, double* gth, cudaStream_t s) {
  k_accum_q<<<1, 1, 0, s>>>(q, a0, a1, a3, a4, gth);
}

// y += a x (n doubles)
// The reverse step's update of the position adjoint from one adjoint pass (sorted order):
// lx[3 id[s] + k] -= c hw[s].k + a f[s].k (f may be null when a = 0).
__global__ void k_adjoint_update(const dvec4* __restrict__ hw, const dvec4* __restrict__ f,
                                 const int32_t* __restrict__ id, int64_t N, double c, double a,
                                 double* __restrict__ lx) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = id[s];
    const dvec4 h = hw[s];
    double dx = c * h.x, dy = c * h.y, dz = c * h.z;
    if (f) {
      const dvec4 g = f[s];
      dx = fma(a, g.x, dx);
      dy = fma(a, g.y, dy);
      dz = fma(a, g.z, dz);
    }
    lx[3 * p] -= dx;
    lx[3 * p + 1] -= dy;
    lx[3 * p + 2] -= dz;
  }
}
void launch_adjoint_update(const dvec4* hw, const dvec4* f, const int32_t* id, int64_t N, double c, double a,
                           double* lx, cudaStream_t s) {
  k_adjoint_update<<<grid_of(N), 256, 0, s>>>(hw, f, id, N, c, a, lx);
}

__global__ void k_axpy(double* __restrict__ y, double a, const double* __restrict__ x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], y[i]);
}
void launch_axpy(double* y, double a, const double* x, int64_t n, cudaStream_t s) {
  k_axpy<<<grid_of(n), 256, 0, s>>>(y, a, x, n);
}

// y = a (u - w) (n doubles)
__global__ void k_scaled_diff(double* __restrict__ y, double a, const double* __restrict__ u,
                              const double* __restrict__ w, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * (u[i] - w[i]);
}
void launch_scaled_diff(double* y, double a, const double* u, const double* w, int64_t n, cudaStream_t s) {
  k_scaled_diff<<<grid_of(n), 256, 0, s>>>(y, a, u, w, n);
}

// Per-block partial sums of (u - w)^2 over n doubles (fixed grid, fixed order).
__global__ void k_sqdiff(const double* __restrict__ u, const double* __restrict__ w, int64_t n,
                         double* __restrict__ part) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = u[i] - w[i];
    acc = fma(d, d, acc);
  }
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}
int launch_sqdiff(const double* u, const double* w, int64_t n, double* part, cudaStream_t s) {
  const int nb = red_blocks(n);
  k_sqdiff<<<nb, kRedThreads, 0, s>>>(u, w, n, part);
  return nb;
}

}  // namespace ljmd
