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
//   partition       a stable counting sort of the batch by shard: each key's
//                   sorted position (written in batch order), the keys (and
//                   values) in sorted order, and the count of each shard;
//   unpermute       results that come back in sorted order are gathered into
//                   the caller's order (out[i] = in[pos[i]]: the writes are in
//                   batch order, the reads walk the shards' runs).
//
// Stability keeps each source's keys in batch order at the owner, so that
// duplicate keys resolve as in one batch (the last value wins).
#include "api_internal.h"

using namespace ckpp;

namespace {

constexpr int kPartThreads = 256;
constexpr int kPartWarps = kPartThreads / 32;
constexpr int kKeysPerThread = 16;
constexpr uint64_t kTile = (uint64_t)kPartThreads * kKeysPerThread;  // keys per block: 4096

__device__ __forceinline__ uint32_t shard_of(const Key& k, uint64_t seed, uint32_t n_shards) {
  const uint64_t h1 = hash_key(k, seed);
  return (uint32_t)((((h1 >> 16) & 0xFFFFull) * n_shards) >> 16);
}

__device__ __forceinline__ Key load_key16(const uint8_t* keys, uint64_t i) {
  const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(keys + 16 * i);
  return Key{v.x, v.y};
}

// Per block (one tile of kTile keys): the number of its keys in each shard,
// shard-major (counts[shard * n_blocks + block]). Each warp adds its lanes of
// one shard with a single shared-memory atomic.
__global__ void __launch_bounds__(kPartThreads) shard_count_kernel(const uint8_t* __restrict__ keys, uint64_t n,
                                                                   uint64_t seed, uint32_t n_shards,
                                                                   uint32_t* __restrict__ counts) {
  __shared__ uint32_t hist[CKPP_MAX_SHARDS];
  for (uint32_t s = threadIdx.x; s < n_shards; s += blockDim.x) hist[s] = 0;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t base = blockIdx.x * kTile;
#pragma unroll 4
  for (int r = 0; r < kKeysPerThread; ++r) {
    const uint64_t i = base + (uint64_t)r * kPartThreads + threadIdx.x;
    const uint32_t s = i < n ? shard_of(load_key16(keys, i), seed, n_shards) : 0xFFFFFFFFu;
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, s);
    if (s != 0xFFFFFFFFu && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&hist[s], (uint32_t)__popc(peers));
  }
  __syncthreads();
  for (uint32_t s = threadIdx.x; s < n_shards; s += blockDim.x) counts[(uint64_t)s * gridDim.x + blockIdx.x] = hist[s];
}

// One block: exclusive scan of the shard-major block counts (in place), and
// the total of each shard. Each thread scans kScanItems consecutive counts per
// pass (loaded together), so a pass covers 1024 x kScanItems counts.
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;

__global__ void __launch_bounds__(kScanThreads) shard_scan_kernel(uint32_t* __restrict__ counts, uint64_t len,
                                                                  uint32_t n_blocks, uint64_t* __restrict__ shard_totals,
                                                                  uint32_t n_shards) {
  __shared__ uint32_t warp_sums[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint64_t base = 0; base < len; base += (uint64_t)kScanThreads * kScanItems) {
    const uint64_t j0 = base + (uint64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems], sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      v[k] = j0 + k < len ? counts[j0 + k] : 0u;
      sum += v[k];
    }
    uint32_t x = sum;  // inclusive warp scan of the threads' sums
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
      if (lane >= d) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = lane < (kScanThreads >> 5) ? warp_sums[lane] : 0u;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, d);
        if (lane >= d) w += y;
      }
      warp_sums[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    uint32_t before = carry + (warp ? warp_sums[warp - 1] : 0u) + x - sum;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      if (j0 + k < len) counts[j0 + k] = before;
      before += v[k];
    }
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) carry = before;  // the last thread's end is the pass's total
    __syncthreads();
  }
  // shard s starts at counts[s * n_blocks]; its total runs to the next shard's start
  for (uint32_t s = threadIdx.x; s < n_shards; s += blockDim.x) {
    const uint64_t start = counts[(uint64_t)s * n_blocks];
    const uint64_t end = (s + 1 < n_shards) ? counts[(uint64_t)(s + 1) * n_blocks] : carry;
    shard_totals[s] = end - start;
  }
}

// Per block (one tile, in rounds of kPartThreads keys): each key's sorted
// position = its block's offset in its shard + the keys of the same shard in
// the tile's earlier rounds + those of earlier warps in this round + its rank
// among its warp's peers, so the sort is stable.
__global__ void __launch_bounds__(kPartThreads) shard_scatter_kernel(
    const uint8_t* __restrict__ keys, const uint64_t* __restrict__ vals, uint64_t n, uint64_t seed, uint32_t n_shards,
    const uint32_t* __restrict__ offsets, uint32_t* __restrict__ pos_of, uint8_t* __restrict__ out_keys,
    uint64_t* __restrict__ out_vals) {
  __shared__ uint32_t warp_count[kPartWarps][CKPP_MAX_SHARDS];
  __shared__ uint32_t next[CKPP_MAX_SHARDS];  // the tile's next position in each shard
  for (uint32_t s = threadIdx.x; s < n_shards; s += blockDim.x) next[s] = offsets[(uint64_t)s * gridDim.x + blockIdx.x];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t base = blockIdx.x * kTile;
  for (int r = 0; r < kKeysPerThread; ++r) {
    if (base + (uint64_t)r * kPartThreads >= n) break;  // uniform over the block
    for (uint32_t j = threadIdx.x; j < kPartWarps * n_shards; j += blockDim.x) warp_count[j / n_shards][j % n_shards] = 0;
    __syncthreads();
    const uint64_t i = base + (uint64_t)r * kPartThreads + threadIdx.x;
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
    if (act) {
      uint32_t before = 0;
      for (uint32_t w = 0; w < warp; ++w) before += warp_count[w][s];
      const uint64_t pos = (uint64_t)next[s] + before + rank;
      pos_of[i] = (uint32_t)pos;
      *reinterpret_cast<ulonglong2*>(out_keys + 16 * pos) = make_ulonglong2(k.k0, k.k1);
      if (vals) out_vals[pos] = vals[i];
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < n_shards; t += blockDim.x) {
      uint32_t add = 0;
      for (uint32_t w = 0; w < kPartWarps; ++w) add += warp_count[w][t];
      next[t] += add;
    }
    __syncthreads();  // the counts are read before the next round clears them
  }
}

__global__ void __launch_bounds__(256) unpermute_kernel(const uint32_t* __restrict__ pos, uint64_t n,
                                                        const uint64_t* __restrict__ in_u64,
                                                        const uint8_t* __restrict__ in_u8,
                                                        uint64_t* __restrict__ out_u64, uint8_t* __restrict__ out_u8) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t p = pos[i];
  if (in_u64) out_u64[i] = in_u64[p];
  if (in_u8) out_u8[i] = in_u8[p];
}

uint64_t part_blocks(uint64_t n) { return (n + kTile - 1) / kTile; }

}  // namespace

extern "C" {

size_t ckpp_shard_workspace_bytes(uint64_t n, uint32_t n_shards) {
  if (n > kMaxBatch || n_shards == 0 || n_shards > CKPP_MAX_SHARDS) return 0;
  return api::align_up(4 * part_blocks(n) * n_shards + 4, api::kAlign);
}

int ckpp_shard_partition(const ckpp_key* keys, const uint64_t* vals, uint64_t n, uint64_t seed, uint32_t n_shards,
                         uint32_t* out_pos, ckpp_key* out_keys, uint64_t* out_vals, uint64_t* out_counts,
                         void* workspace, size_t workspace_bytes, ckpp_stream_t stream) {
  if (api::check_keys(keys, n) || n_shards == 0 || n_shards > CKPP_MAX_SHARDS || !out_counts ||
      !api::aligned(out_counts, 8))
    return CKPP_EINVAL;
  if (n && (!out_pos || !out_keys || !api::aligned(out_keys, 16) || !api::aligned(out_pos, 4))) return CKPP_EINVAL;
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
  shard_scan_kernel<<<1, kScanThreads, 0, s>>>(counts, blocks * n_shards, (uint32_t)blocks, out_counts, n_shards);
  shard_scatter_kernel<<<(unsigned)blocks, kPartThreads, 0, s>>>(k8, vals, n, seed, n_shards, counts, out_pos,
                                                                  reinterpret_cast<uint8_t*>(out_keys), out_vals);
  return api::cuda_rc(cudaGetLastError());
}

int ckpp_shard_unpermute(const uint32_t* pos, uint64_t n, const uint64_t* in_u64, const uint8_t* in_u8,
                         uint64_t* out_u64, uint8_t* out_u8, ckpp_stream_t stream) {
  if (n > kMaxBatch || (n && !pos) || (in_u64 == nullptr) != (out_u64 == nullptr) ||
      (in_u8 == nullptr) != (out_u8 == nullptr))
    return CKPP_EINVAL;
  if ((in_u64 && (!api::aligned(in_u64, 8) || !api::aligned(out_u64, 8))) || !api::aligned(pos, 4))
    return CKPP_EINVAL;
  if (!n) return CKPP_OK;
  unpermute_kernel<<<(unsigned)((n + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      pos, n, in_u64, in_u8, out_u64, out_u8);
  return api::cuda_rc(cudaGetLastError());
}

}  // extern "C"
