// Velocity-Verlet (the benchmark's second-order symplectic integrator, Sec. 4.5), fused:
//
//   v_full = v + kpre F          (completes the previous step; its kinetic energy is taken)
//   v     <- v + (kpre + kpost) F (the first half-kick of the next step folded in)
//   x     <- x + dt v             (drift)
//
// then the force kernel's copy of the positions is rewritten (mixed form: the 32-bit fixed-point
// records, X = round(x_state / u) mod 2^32 with u = 2^-qk and the sorted index in w; FP64 form: a
// dvec4 copy) and the displacement since the last list construction is reduced (device-wide max)
// for the margin/2 validity rule.
// State x, v is FP64 (positions stored as offset + x).  Per component the FP64 pipe does two
// FMAs; the kinetic energy of the mixed form is taken in FP32 per particle and summed in FP64.
// In the mixed form every FP32 <-> FP64 conversion is done with integer operations (exact for
// FP32 -> FP64, rounded to nearest for FP64 -> FP32), which keeps the FP64 pipe for the seven
// operations per particle that need it.
#include "common.cuh"

namespace ljmd {

// The list-validity decision of a device-decided run (the host rule of ljmd_step, taken on the
// device so that steps follow each other without a host round trip): the largest squared
// displacement and drift speed of the step are taken (and reset for the next one); with the
// margin/2 rule the list expired when the displacement exceeds the limit, with DUTC when the
// remaining buffer, less the closing 2 v_max dt of the step, is used up.  An expired list stops
// the run at step s.  One thread.
__device__ __forceinline__ void step_check_one(uint32_t* dmax_bits, StepCtl* ctl, int s, double disp_limit, int dutc,
                                               double two_dt) {
  if (ctl->stop) return;
  const float d2 = __uint_as_float(atomicExch(dmax_bits, 0u)), v2 = __uint_as_float(atomicExch(dmax_bits + 1, 0u));
  ctl->last[0] = d2;
  ctl->last[1] = v2;
  bool expired;
  if (dutc) {
    const double b = ctl->dutc - two_dt * sqrt((double)v2) * (1.0 + 1e-6);
    ctl->dutc = b;
    expired = !(b > 0.0);
  } else {
    expired = sqrt((double)d2) > disp_limit;
  }
  if (expired) {
    ctl->stop = 1;
    ctl->stop_at = s;
  }
}

// One particle's inputs to the integrator: force, velocity, position and (when the position copy is
// rewritten) the displacement reference.
template <bool MIXED>
struct IntegrateIn;
template <>
struct IntegrateIn<true> {
  float4 f;
  uint4 r;
  double v[3], x[3];
};
template <>
struct IntegrateIn<false> {
  dvec4 f, r;
  double v[3], x[3];
};

template <bool MIXED>
__device__ __forceinline__ void integrate_load(IntegrateIn<MIXED>& in, const double* __restrict__ x,
                                               const double* __restrict__ v, const void* __restrict__ fptr,
                                               const void* __restrict__ refp, int64_t N, int64_t i, int shadow) {
  if constexpr (MIXED) {
    in.f = ((const float4*)fptr)[i];
    if (shadow) in.r = ((const uint4*)refp)[i];
  } else {
    in.f = ((const dvec4*)fptr)[i];
    if (shadow) in.r = ((const dvec4*)refp)[i];
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    in.v[k] = v[k * N + i];
    in.x[k] = x[k * N + i];
  }
}

// Hint that the lines holding particle j's inputs be brought into L2 (one prefetch per stream; no
// registers are held for the data).
template <bool MIXED>
__device__ __forceinline__ void integrate_prefetch_l2(const double* x, const double* v, const void* fptr,
                                                      const void* refp, int64_t N, int64_t j, int shadow) {
  const void* f = MIXED ? (const void*)((const float4*)fptr + j) : (const void*)((const dvec4*)fptr + j);
  asm volatile("prefetch.global.L2 [%0];" ::"l"(f));
  if (shadow) {
    const void* r = MIXED ? (const void*)((const uint4*)refp + j) : (const void*)((const dvec4*)refp + j);
    asm volatile("prefetch.global.L2 [%0];" ::"l"(r));
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(v + k * N + j));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(x + k * N + j));
  }
}

// The grid-stride loop is software-pipelined: the next particle's loads are issued before the
// FP64 kick and drift of the current one, so that the FP64 pipe (7 operations per particle at
// 1/64 of the FP32 rate) works while those loads are in flight instead of after them, and the lines
// of the particle kPrefetchAhead strides on are requested into L2, which keeps more of HBM's
// requests in flight than the registers of two particles per thread can.
constexpr int kPrefetchAhead = 2;

template <bool MIXED>
__global__ void __launch_bounds__(256) k_integrate(double* __restrict__ x, double* __restrict__ v,
                                                   const void* __restrict__ fptr, void* __restrict__ pos,
                                                   const void* __restrict__ refp, int64_t N, IntegrateArgs a,
                                                   double* __restrict__ ke_part, uint32_t* __restrict__ dmax_bits,
                                                   int32_t* __restrict__ status, StepFinish fin,
                                                   const int* __restrict__ skip) {
  if (skip && *skip) return;  // a device-decided run stopped before this step
  const float qu = __int_as_float((127 - a.qk) << 23);  // u = 2^-qk
  const double kk = a.kpre + a.kpost;
  const float kpre_f = (float)a.kpre;
  double ke_acc = 0.0;
  float d2max = 0.0f, v2max = 0.0f;
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  IntegrateIn<MIXED> cur = {};
  if (i < N) integrate_load<MIXED>(cur, x, v, fptr, refp, N, i, a.shadow);
  for (; i < N; i += stride) {
    IntegrateIn<MIXED> nxt = {};
    if (i + stride < N) integrate_load<MIXED>(nxt, x, v, fptr, refp, N, i + stride, a.shadow);
    if (i + kPrefetchAhead * stride < N)
      integrate_prefetch_l2<MIXED>(x, v, fptr, refp, N, i + kPrefetchAhead * stride, a.shadow);
    double F[3];
    float Ff[3] = {0.0f, 0.0f, 0.0f};
    if constexpr (MIXED) {
      const float4 f = cur.f;
      Ff[0] = f.x;
      Ff[1] = f.y;
      Ff[2] = f.z;
      F[0] = f32_to_f64(f.x);
      F[1] = f32_to_f64(f.y);
      F[2] = f32_to_f64(f.z);
    } else {
      const dvec4 f = cur.f;
      F[0] = f.x;
      F[1] = f.y;
      F[2] = f.z;
    }
    double xs[3];
    float ke_i = 0.0f, vd2 = 0.0f;
    double ke_d = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double vk = cur.v[k];
      if (a.ke) {
        if (MIXED) {
          const float vf = fmaf(kpre_f, Ff[k], f64_to_f32(vk));
          ke_i = fmaf(vf, vf, ke_i);
        } else {
          const double vf = fma(a.kpre, F[k], vk);
          ke_d = fma(vf, vf, ke_d);
        }
      }
      if (kk != 0.0) vk = fma(kk, F[k], vk);
      if (a.speed) {
        const float vs = MIXED ? f64_to_f32(vk) : (float)vk;
        vd2 = fmaf(vs, vs, vd2);
      }
      double xk = cur.x[k];
      if (a.dt != 0.0) xk = fma(a.dt, vk, xk);
      v[k * N + i] = vk;
      x[k * N + i] = xk;
      xs[k] = xk;
      bad |= !finite_d(xk) || !finite_d(vk);
    }
    if (MIXED) ke_acc += f32_to_f64(0.5f * ke_i);  // exact halving and conversion, one FP64 add
    else ke_acc += 0.5 * ke_d;
    if (a.shadow) {
      // speed of the drift (the velocity that moved the particle this step), for the DUTC rule
      v2max = fmaxf(v2max, vd2);
      if constexpr (MIXED) {
        const uint4 q = make_uint4(fixq(xs[0], a.qk), fixq(xs[1], a.qk), fixq(xs[2], a.qk), (uint32_t)i);
        ((uint4*)pos)[i] = q;
        // displacement since the list was built, from the records: exact integer differences
        // (within u of the FP64 ones), converted once and scaled by u
        const uint4 r = cur.r;
        const float dx = qdiff(q.x, r.x) * qu, dy = qdiff(q.y, r.y) * qu, dz = qdiff(q.z, r.z) * qu;
        d2max = fmaxf(d2max, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
      } else {
        ((dvec4*)pos)[i] = make_dvec4(xs[0], xs[1], xs[2], 0.0);
        const dvec4 r = cur.r;
        const double dx = xs[0] - r.x, dy = xs[1] - r.y, dz = xs[2] - r.z;
        // rounded up to FP32, so the measured maximum never falls short of the FP64 value and the
        // margin/2 rule keeps its guarantee at the FP64 form's tight limit
        d2max = fmaxf(d2max, __double2float_ru(fma(dx, dx, fma(dy, dy, dz * dz))));
      }
    }
    cur = nxt;
  }
  if (bad) atomicOr(status, LJ_ST_NONFINITE);
  __shared__ double sh[32];
  __shared__ float shf[32];
  const double tk = block_sum(ke_acc, sh);
  if (threadIdx.x == 0 && a.ke) ke_part[blockIdx.x] = tk;
  if (a.shadow && !a.speed) {
    const float m = block_max(d2max, shf);
    if (threadIdx.x == 0) atomicMax(dmax_bits, __float_as_uint(m));
  } else if (a.shadow) {  // both maxima in one pass over the warps
    __shared__ float shv[32];
    d2max = warp_max(d2max);
    v2max = warp_max(v2max);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) {
      shf[w] = d2max;
      shv[w] = v2max;
    }
    __syncthreads();
    if (w == 0) {
      const bool in = l < (int)(blockDim.x >> 5);
      const float md = warp_max(in ? shf[l] : 0.0f), mv = warp_max(in ? shv[l] : 0.0f);
      if (l == 0) {
        atomicMax(dmax_bits, __float_as_uint(md));
        atomicMax(dmax_bits + 1, __float_as_uint(mv));
      }
    }
  }
  if (fin.ticket) {  // the last CTA to finish takes the energy record and the validity check
    // thread 0 wrote the CTA's partial (the maxima went by device-wide atomics): it alone orders
    // that write before its ticket
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      s_last = atomicAdd(fin.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      if (fin.rec)
        energy_record_block(fin.pv, fin.nbf, ke_part, gridDim.x, fin.pe_scale, fin.energies, fin.log, fin.cap,
                            fin.count, fin.step);
      if (threadIdx.x == 0) {
        if (fin.check) step_check_one(dmax_bits, fin.ctl, fin.s, fin.disp_limit, fin.dutc, fin.two_dt);
        *fin.ticket = 0u;
      }
    }
  }
}

// Block shape: 256-thread blocks of one resident wave (at most red_blocks(N)), so that the grid-stride
// loop ends in step on every SM; for a system too small to give every SM a block, narrower blocks
// (down to one warp) spread the particles over the SMs, each of whose FP64 pipes takes 1/64 of the
// FP32 rate.
template <bool MIXED>
static void integrate_shape(int64_t N, int& blocks, int& threads) {
  static int per_sm = 0, sms = 0;
  if (per_sm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_integrate<MIXED>, kRedThreads, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  }
  threads = kRedThreads;
  while (threads > 32 && (N + threads - 1) / threads < sms) threads >>= 1;
  if (threads == kRedThreads) {
    const int b = red_blocks(N);
    blocks = b < per_sm * sms ? b : per_sm * sms;
  } else {
    const int64_t b = (N + threads - 1) / threads;  // below 2 sms: within the partial arrays
    blocks = (int)(b < 1 ? 1 : b);
  }
}

int launch_integrate(int precision, double* x, double* v, const void* f, void* pos, const void* ref, int64_t N,
                     IntegrateArgs a, double* ke_part, uint32_t* dmax_bits, int32_t* status, StepFinish fin,
                     cudaStream_t s, const int* skip) {
  int blocks = 1, threads = kRedThreads;
  if (precision == LJ_MIXED) {
    integrate_shape<true>(N, blocks, threads);
    k_integrate<true><<<blocks, threads, 0, s>>>(x, v, f, pos, ref, N, a, ke_part, dmax_bits, status, fin, skip);
  } else {
    integrate_shape<false>(N, blocks, threads);
    k_integrate<false><<<blocks, threads, 0, s>>>(x, v, f, pos, ref, N, a, ke_part, dmax_bits, status, fin, skip);
  }
  return blocks;
}

// Position copies for the force and list kernels from the FP64 state (no integration): the FP32
// hi parts always, with the sorted index in w (the list construction filters on them in both
// forms); for the mixed form the fixed-point records, for FP64 the dvec4 copy; and the
// displacement reference (the records for mixed, the dvec4 for FP64) if ref != NULL.
__global__ void k_shadow(const double* __restrict__ x, int64_t N, int mixed, int qk, float4* __restrict__ hi,
                         uint4* __restrict__ xq, dvec4* __restrict__ pos64, void* __restrict__ ref,
                         const int* __restrict__ pred) {
  if (pred && !*pred) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double a = x[i], b = x[N + i], c = x[2 * N + i];
    float4 h;
    float unused;
    split_hi_lo(a, h.x, unused);
    split_hi_lo(b, h.y, unused);
    split_hi_lo(c, h.z, unused);
    h.w = __int_as_float((int)i);  // the sorted index, for the list construction
    hi[i] = h;
    if (mixed) {
      const uint4 q = make_uint4(fixq(a, qk), fixq(b, qk), fixq(c, qk), (uint32_t)i);
      xq[i] = q;
      if (ref) ((uint4*)ref)[i] = q;
    } else {
      pos64[i] = make_dvec4(a, b, c, 0.0);
      if (ref) ((dvec4*)ref)[i] = make_dvec4(a, b, c, 0.0);
    }
  }
}

void launch_shadow_all(const double* x, int64_t N, int mixed, int qk, float4* hi, uint4* xq, dvec4* pos64, void* ref,
                       cudaStream_t s, const int* pred) {
  int64_t b = (N + 255) / 256;
  if (b < 1) b = 1;
  k_shadow<<<(int)(b < 1048576 ? b : 1048576), 256, 0, s>>>(x, N, mixed, qk, hi, xq, pos64, ref, pred);
}

}  // namespace ljmd
