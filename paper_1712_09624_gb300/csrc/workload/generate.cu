// Device-side synthetic traffic: the inputs of workload.py, drawn in place.
// Philox4x64-10 is written from its definition (Salmon et al., SC'11): ten
// rounds of two 64x64->128 multiplications with the round keys bumped by the
// Weyl constants between rounds.
#include <cstdint>
#include <cuda_runtime.h>

#include "../../../include/ckpp_workload.h"

namespace {

constexpr uint64_t kM0 = 0xD2E7470EE14C6C93ull, kM1 = 0xCA5A826395121157ull;
constexpr uint64_t kW0 = 0x9E3779B97F4A7C15ull, kW1 = 0xBB67AE8584CAA73Bull;
constexpr uint64_t kStreamInsert = 1, kStreamNegative = 2, kStreamNegMask = 3, kStreamPosPick = 4;

struct Block {
  uint64_t w[4];
};

__device__ __forceinline__ Block philox4x64_10(uint64_t c0, uint64_t k0, uint64_t k1) {
  uint64_t x0 = c0, x1 = 0, x2 = 0, x3 = 0;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t hi0 = __umul64hi(kM0, x0), lo0 = kM0 * x0;
    const uint64_t hi1 = __umul64hi(kM1, x2), lo1 = kM1 * x2;
    const uint64_t n0 = hi1 ^ x1 ^ k0, n2 = hi0 ^ x3 ^ k1;
    x0 = n0;
    x1 = lo1;
    x2 = n2;
    x3 = lo0;
    k0 += kW0;
    k1 += kW1;
  }
  return Block{{x0, x1, x2, x3}};
}

// Raw outputs 2i and 2i+1 of stream (seed, s): one half of a Philox block.
__device__ __forceinline__ void raw_pair(uint64_t seed, uint64_t s, uint64_t i, uint64_t& a, uint64_t& b) {
  const Block blk = philox4x64_10(i / 2 + 1, seed, s);
  a = (i & 1) ? blk.w[2] : blk.w[0];
  b = (i & 1) ? blk.w[3] : blk.w[1];
}

__device__ __forceinline__ uint64_t raw_one(uint64_t seed, uint64_t s, uint64_t t) {
  const Block blk = philox4x64_10(t / 4 + 1, seed, s);
  return blk.w[t & 3];
}

// Key i of stream (seed, s): src|dst from the first word; ports from the low
// half of the second, protocol 6 or 17 from its bit 32.
__device__ __forceinline__ void make_key(uint64_t seed, uint64_t s, uint64_t i, uint64_t& k0, uint64_t& k1) {
  uint64_t r0, r1;
  raw_pair(seed, s, i, r0, r1);
  k0 = r0;
  const uint64_t proto = ((r1 >> 32) & 1) ? 17ull : 6ull;
  k1 = (r1 & 0xFFFFFFFFull) | (proto << 32);
}

__global__ void fill_kernel(uint64_t seed, uint64_t first, uint64_t n, uint8_t* keys, uint64_t* vals) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t k0, k1;
  make_key(seed, kStreamInsert, first + i, k0, k1);
  reinterpret_cast<ulonglong2*>(keys)[i] = make_ulonglong2(k0, k1);
  if (vals) vals[i] = first + i;
}

__global__ void keys_at_kernel(uint64_t seed, const uint64_t* __restrict__ idx, uint64_t n, uint8_t* keys) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t k0, k1;
  make_key(seed, kStreamInsert, idx[i], k0, k1);
  reinterpret_cast<ulonglong2*>(keys)[i] = make_ulonglong2(k0, k1);
}

__global__ void lookup_batch_kernel(uint64_t seed, uint64_t batch_id, uint64_t n, uint64_t m, double neg_rate,
                                    uint8_t* keys, uint8_t* found, uint64_t* value) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t sub = (seed << 20) ^ batch_id;
  const uint64_t u = raw_one(sub, kStreamNegMask, i);
  const bool neg = m == 0 || (double)(u >> 11) * 0x1p-53 < neg_rate;
  uint64_t k0, k1, pick = 0;
  if (neg) {
    make_key(sub, kStreamNegative, i, k0, k1);
  } else {
    pick = ((raw_one(sub, kStreamPosPick, i) >> 32) * m) >> 32;
    make_key(seed, kStreamInsert, pick, k0, k1);
  }
  reinterpret_cast<ulonglong2*>(keys)[i] = make_ulonglong2(k0, k1);
  if (found) found[i] = neg ? 0 : 1;
  if (value) value[i] = neg ? 0 : pick;
}

}  // namespace

extern "C" int ckpp_wl_fill_keys(uint64_t seed, uint64_t first, uint64_t n, uint8_t* out_keys, uint64_t* out_vals,
                                 ckpp_wl_stream_t stream) {
  if (n == 0) return 0;
  if (!out_keys || reinterpret_cast<uintptr_t>(out_keys) % 16 || (out_vals && reinterpret_cast<uintptr_t>(out_vals) % 8))
    return -1;
  fill_kernel<<<(unsigned)((n + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(seed, first, n, out_keys,
                                                                                                 out_vals);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

extern "C" int ckpp_wl_keys_at(uint64_t seed, const uint64_t* idx, uint64_t n, uint8_t* out_keys,
                               ckpp_wl_stream_t stream) {
  if (n == 0) return 0;
  if (!idx || !out_keys || reinterpret_cast<uintptr_t>(out_keys) % 16 || reinterpret_cast<uintptr_t>(idx) % 8)
    return -1;
  keys_at_kernel<<<(unsigned)((n + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(seed, idx, n,
                                                                                                   out_keys);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

extern "C" int ckpp_wl_lookup_batch(uint64_t seed, uint64_t batch_id, uint64_t n, uint64_t n_inserted,
                                    double neg_rate, uint8_t* out_keys, uint8_t* expect_found,
                                    uint64_t* expect_value, ckpp_wl_stream_t stream) {
  if (n == 0) return 0;
  if (!out_keys || reinterpret_cast<uintptr_t>(out_keys) % 16 || n_inserted >= (1ull << 32) ||
      (expect_value && reinterpret_cast<uintptr_t>(expect_value) % 8))
    return -1;
  lookup_batch_kernel<<<(unsigned)((n + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      seed, batch_id, n, n_inserted, neg_rate, out_keys, expect_found, expect_value);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
