// Hash sharding of a batch across the ranks of a multi-GPU table: one table
// per GPU, each owning the keys of its shard. The paper's tables are private
// to one core each (Sec. 2 and Sec. 5.3); a table split over GPUs needs every
// key of a batch to reach its owner (an all-to-all of keys), the owner's
// ordinary bulk call, and the results' way back (a second all-to-all). These
// kernels are the device half of that exchange:
//
//   shard of a key  ((H1 >> 16) & 0xFFFF) * n_shards >> 16: bits 16-31 of the
//                   primary hash, which neither the tag (bits 0-15) nor the
//                   primary bucket (bits 32-63) uses, so every shard's table
//                   sees uniform buckets and tags;
//   partition       a stable counting sort of the batch by shard: the order
//                   (original index of each sorted position), the keys (and
//                   values) in that order, and the count of each shard;
//   unpermute       results that come back in sorted order are written to
//                   the caller's order.
//
// Stability keeps each source's keys in batch order at the owner, so that
// duplicate keys resolve as in one batch (the last value wins).
#include "api_internal.h"

using namespace ckpp;

namespace {

constexpr int kPartThreads = 256;  // keys per block
constexpr int kPartWarps = kPartThreads / 32;

__device__ __forceinline__ uint32_t shard_of(const Key& k, uint64_t seed, uint32_t n_shards) {
  const uint64_t h1 = hash_key(k, seed);
  return (uint32_t)((((h1 >> 16) & 0xFFFFull) * n_shards) >> 16);
}

__device__ __forceinline__ Key load_key16(const uint8_t* keys, uint64_t i) {
  const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(keys + 16 * i);
  return Key{v.x, v.y};
}

// Per block: the number of its keys in each shard, shard-major
// (counts[shard * n_blocks + block]).
__global__ void __launch_bounds__(kPartThreads) shard_count_kernel(const uint8_t* __restrict__ keys, uint64_t n,
                                                                   uint64_t seed, uint32_t n_shards,
                                                                   uint32_t* __restrict__ counts) {
  __shared__ uint32_t hist[CKPP_MAX_SHARDS];
  for (uint32_t s = threadIdx.x; s < n_shards; s += blockDim.x) hist[s] = 0;
  __syncthreads();
  const uint64_t i = blockIdx.x * (uint64_t)kPartThreads + threadIdx.x;
  if (i < n) atomicAdd(&hist[shard_of(load_key16(keys, i), seed, n_shards)], 1u);
  __syncthreads();
  for (uint32_t s = threadIdx.x; s < n_shards; s += blockDim.x) counts[(uint64_t)s * gridDim.x + blockIdx.x] = hist[s];
}

// One block: exclusive scan of the shard-major block counts (in place), and
// the total of each shard.
__global__ void __launch_bounds__(1024) shard_scan_kernel(uint32_t* __restrict__ counts, uint64_t len,
                                                          uint32_t n_blocks, uint64_t* __restrict__ shard_totals,
                                                          uint32_t n_shards) {
  __shared__ uint32_t warp_sums[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint64_t base = 0; base < len; base += blockDim.x) {
    const uint64_t j = base + threadIdx.x;
    const uint32_t v = j < len ? counts[j] : 0u;
    uint32_t x = v;  // inclusive warp scan
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
      if (lane >= d) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = lane < (blockDim.x >> 5) ? warp_sums[lane] : 0u;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, d);
        if (lane >= d) w += y;
      }
      warp_sums[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const uint32_t before = carry + (warp ? warp_sums[warp - 1] : 0u) + x - v;
    if (j < len) counts[j] = before;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + v;
    __syncthreads();
  }
  // shard s starts at counts[s * n_blocks]; its total runs to the next shard's start
  for (uint32_t s = threadIdx.x; s < n_shards; s += blockDim.x) {
    const uint64_t start = counts[(uint64_t)s * n_blocks];
    const uint64_t end = (s + 1 < n_shards) ? counts[(uint64_t)(s + 1) * n_blocks] : carry;
    shard_totals[s] = end - start;
  }
}

// Per block: each key's sorted position = its block's offset in its shard +
// the keys of the same shard before it in the block (warp ballots, then the
// earlier warps' counts), so the sort is stable.
__global__ void __launch_bounds__(kPartThreads) shard_scatter_kernel(
    const uint8_t* __restrict__ keys, const uint64_t* __restrict__ vals, uint64_t n, uint64_t seed, uint32_t n_shards,
    const uint32_t* __restrict__ offsets, uint32_t* __restrict__ order, uint8_t* __restrict__ out_keys,
    uint64_t* __restrict__ out_vals) {
  __shared__ uint32_t warp_count[kPartWarps][CKPP_MAX_SHARDS];
  for (uint32_t j = threadIdx.x; j < kPartWarps * n_shards; j += blockDim.x)
    warp_count[j / n_shards][j % n_shards] = 0;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t i = blockIdx.x * (uint64_t)kPartThreads + threadIdx.x;
  const bool act = i < n;
  Key k{0, 0};
  uint32_t s = 0xFFFFFFFFu;  // inactive lanes form their own group
  if (act) {
    k = load_key16(keys, i);
    s = shard_of(k, seed, n_shards);
  }
  const uint32_t peers = __match_any_sync(0xFFFFFFFFu, s);
  const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
  if (act && rank == 0) warp_count[warp][s] = __popc(peers);
  __syncthreads();
  if (!act) return;
  uint32_t before = 0;
  for (uint32_t w = 0; w < warp; ++w) before += warp_count[w][s];
  const uint64_t pos = (uint64_t)offsets[(uint64_t)s * gridDim.x + blockIdx.x] + before + rank;
  order[pos] = (uint32_t)i;
  *reinterpret_cast<ulonglong2*>(out_keys + 16 * pos) = make_ulonglong2(k.k0, k.k1);
  if (vals) out_vals[pos] = vals[i];
}

__global__ void __launch_bounds__(256) unpermute_kernel(const uint32_t* __restrict__ order, uint64_t n,
                                                        const uint64_t* __restrict__ in_u64,
                                                        const uint8_t* __restrict__ in_u8,
                                                        uint64_t* __restrict__ out_u64, uint8_t* __restrict__ out_u8) {
  const uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  const uint32_t i = order[j];
  if (in_u64) out_u64[i] = in_u64[j];
  if (in_u8) out_u8[i] = in_u8[j];
}

uint64_t part_blocks(uint64_t n) { return (n + kPartThreads - 1) / kPartThreads; }

}  // namespace

extern "C" {

size_t ckpp_shard_workspace_bytes(uint64_t n, uint32_t n_shards) {
  if (n > kMaxBatch || n_shards == 0 || n_shards > CKPP_MAX_SHARDS) return 0;
  return api::align_up(4 * part_blocks(n) * n_shards + 4, api::kAlign);
}

int ckpp_shard_partition(const ckpp_key* keys, const uint64_t* vals, uint64_t n, uint64_t seed, uint32_t n_shards,
                         uint32_t* out_order, ckpp_key* out_keys, uint64_t* out_vals, uint64_t* out_counts,
                         void* workspace, size_t workspace_bytes, ckpp_stream_t stream) {
  if (api::check_keys(keys, n) || n_shards == 0 || n_shards > CKPP_MAX_SHARDS || !out_counts ||
      !api::aligned(out_counts, 8))
    return CKPP_EINVAL;
  if (n && (!out_order || !out_keys || !api::aligned(out_keys, 16) || !api::aligned(out_order, 4))) return CKPP_EINVAL;
  if ((vals == nullptr) != (out_vals == nullptr)) return CKPP_EINVAL;
  if (vals && (!api::aligned(vals, 8) || !api::aligned(out_vals, 8))) return CKPP_EINVAL;
  if (!workspace || workspace_bytes < ckpp_shard_workspace_bytes(n, n_shards) || !api::aligned(workspace, 4))
    return CKPP_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!n) return api::cuda_rc(cudaMemsetAsync(out_counts, 0, 8ull * n_shards, s));
  const uint64_t blocks = part_blocks(n);
  uint32_t* counts = static_cast<uint32_t*>(workspace);
  const uint8_t* k8 = reinterpret_cast<const uint8_t*>(keys);
  shard_count_kernel<<<(unsigned)blocks, kPartThreads, 0, s>>>(k8, n, seed, n_shards, counts);
  shard_scan_kernel<<<1, 1024, 0, s>>>(counts, blocks * n_shards, (uint32_t)blocks, out_counts, n_shards);
  shard_scatter_kernel<<<(unsigned)blocks, kPartThreads, 0, s>>>(k8, vals, n, seed, n_shards, counts, out_order,
                                                                  reinterpret_cast<uint8_t*>(out_keys), out_vals);
  return api::cuda_rc(cudaGetLastError());
}

int ckpp_shard_unpermute(const uint32_t* order, uint64_t n, const uint64_t* in_u64, const uint8_t* in_u8,
                         uint64_t* out_u64, uint8_t* out_u8, ckpp_stream_t stream) {
  if (n > kMaxBatch || (n && !order) || (in_u64 == nullptr) != (out_u64 == nullptr) ||
      (in_u8 == nullptr) != (out_u8 == nullptr))
    return CKPP_EINVAL;
  if ((in_u64 && (!api::aligned(in_u64, 8) || !api::aligned(out_u64, 8))) || !api::aligned(order, 4))
    return CKPP_EINVAL;
  if (!n) return CKPP_OK;
  unpermute_kernel<<<(unsigned)((n + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      order, n, in_u64, in_u8, out_u64, out_u8);
  return api::cuda_rc(cudaGetLastError());
}

}  // extern "C"
