// Pair-list export into a fixed, statically allocated device scratch array (the allocation-free
// variant of the pair export).  The list is decoded into 64-bit keys (id_a << 32 | id_b, a < b),
// sorted on the device with a bitonic network and copied out; nothing here allocates memory.
#include <mutex>

#include "ljmd_internal.h"

namespace ljmd {

namespace {

constexpr int kHeaderWords = 32;  // 256 bytes ahead of the keys; word 0 holds the kept-pair counter
constexpr int kMaxDevices = 64;

// One scratch per device, shared by every handle and stream of the process.  Concurrent calls
// that use it on the same device race.
__device__ __align__(256) unsigned long long g_pairs_scratch[kHeaderWords + LJ_PAIRS_STATIC_MAX_ENTRIES];

std::mutex g_mu;
unsigned long long* g_addr[kMaxDevices] = {};

// Each decoded list entry (sorted indices of key and partner, or all-ones in tile padding) becomes
// the key (id_a << 32 | id_b) of its pair with id_a < id_b, or all-ones if the entry is padding or
// (full list) the second copy of a pair.  Converted in place: each thread owns one 8-byte slot.
__global__ void k_entries_to_keys(unsigned long long* __restrict__ keys, uint64_t E,
                                  const int32_t* __restrict__ id, int64_t N, int full,
                                  unsigned int* __restrict__ counter, int32_t* __restrict__ status) {
  unsigned int kept = 0;
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < E; k += (uint64_t)gridDim.x * blockDim.x) {
    const uint2 e = reinterpret_cast<const uint2*>(keys)[k];
    unsigned long long key = ~0ull;
    if (e.x != 0xffffffffu || e.y != 0xffffffffu) {
      if (e.x >= (uint64_t)N || e.y >= (uint64_t)N) {
        atomicOr(status, LJ_ST_LIST_OVERFLOW);
      } else {
        const uint32_t a = (uint32_t)id[e.x], b = (uint32_t)id[e.y];
        if (!full || a < b) {
          const uint32_t lo = a < b ? a : b, hi = a < b ? b : a;
          key = ((unsigned long long)lo << 32) | hi;
          kept += 1;
        }
      }
    }
    keys[k] = key;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
  if ((threadIdx.x & 31) == 0 && kept) atomicAdd(counter, kept);
}

// One compare-exchange stage (block size k, partner distance j) of an ascending bitonic sort of
// P = 2^m keys; thread t handles the pair (i, i + j) where i is t with a zero inserted at bit j.
__global__ void k_bitonic_stage(unsigned long long* __restrict__ keys, uint32_t half_P, uint32_t k, uint32_t j) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= half_P) return;
  const uint32_t i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
  const uint32_t l = i | j;
  const bool up = (i & k) == 0;
  const unsigned long long a = keys[i], b = keys[l];
  if ((a > b) == up) {
    keys[i] = b;
    keys[l] = a;
  }
}

}  // namespace

int pairs_static_scratch(int device, unsigned long long** counter_word, unsigned long long** keys) {
  if (device < 0 || device >= kMaxDevices) return LJ_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_pairs_scratch) != cudaSuccess) {
      cudaGetLastError();
      return LJ_EDEVICE;
    }
    g_addr[device] = (unsigned long long*)p;
  }
  *counter_word = g_addr[device];
  *keys = g_addr[device] + kHeaderWords;
  return LJ_OK;
}

void launch_entries_to_keys(unsigned long long* keys, uint64_t E, const int32_t* id, int64_t N, int full,
                            unsigned int* counter, int32_t* status, cudaStream_t s) {
  uint64_t b = (E + 255) / 256;
  if (b > 4096) b = 4096;
  if (b == 0) b = 1;
  k_entries_to_keys<<<(unsigned)b, 256, 0, s>>>(keys, E, id, N, full, counter, status);
}

int launch_bitonic_sort(unsigned long long* keys, uint32_t P, cudaStream_t s) {
  int launches = 0;
  const uint32_t half_P = P / 2;
  const unsigned blocks = (half_P + 255) / 256;
  for (uint32_t k = 2; k <= P; k <<= 1)
    for (uint32_t j = k / 2; j > 0; j >>= 1) {
      k_bitonic_stage<<<blocks, 256, 0, s>>>(keys, half_P, k, j);
      launches += 1;
    }
  return launches;
}

}  // namespace ljmd
