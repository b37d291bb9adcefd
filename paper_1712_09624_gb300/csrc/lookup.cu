// Bulk lookup over one table (Sec. 2 and Sec. 4.1 of the paper): one thread
// per key, the per-key method in probe.cuh.
//
// The paper hides DRAM latency by interleaving the steps of a batch of lookups
// with prefetches (Sec. 3); on the GPU the same memory-level parallelism comes
// from tens of thousands of resident threads, each with its own chain of loads.
// Keys are streamed with coalesced 16-byte loads and results with coalesced
// stores; bucket sectors are read with an L2 evict_last hint (the bucket array
// is the table's hot part), records and keys with evict_first.
#include "probe.cuh"

namespace ckpp {

namespace {

// kHostIO: keys and results live in pinned host memory, reached over
// NVLink-C2C by the loads and stores themselves (no staging copy); such keys
// are read with plain loads, without the read-only path or L2 hints.
template <bool kTimers, bool kCount, bool kHostIO, int kVariant>
__global__ void __launch_bounds__(256) lookup_kernel(TableView t, const uint8_t* __restrict__ keys, uint64_t n,
                                                     uint64_t* __restrict__ out_vals,
                                                     uint8_t* __restrict__ out_found, uint32_t now,
                                                     uint32_t refresh_ttl, unsigned long long* __restrict__ counts) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  uint32_t nsec = 0, nrec = 0, nkey = 0;
  if (i < n) {
    const uint64_t keep = policy_evict_last();
    const uint64_t stream = policy_evict_first();
    Key k;
    if (kHostIO) {
      const ulonglong2 kk = *reinterpret_cast<const ulonglong2*>(keys + 16 * i);
      k = Key{kk.x, kk.y};
    } else {
      k = ld_key_ro(keys + 16 * i, stream);
    }
    uint64_t value;
    const bool found = probe_key<kTimers, kCount, kVariant>(t, k, now, refresh_ttl, keep, stream, value, nsec, nrec);
    if (kCount) {
      nkey = 1;
    } else {
      out_vals[i] = value;
      out_found[i] = found ? 1 : 0;
    }
  }
  if (kCount) {
    nkey = __reduce_add_sync(0xFFFFFFFFu, nkey);
    nsec = __reduce_add_sync(0xFFFFFFFFu, nsec);
    nrec = __reduce_add_sync(0xFFFFFFFFu, nrec);
    if ((threadIdx.x & 31) == 0 && nkey) {
      atomicAdd(counts + 0, (unsigned long long)nkey);
      atomicAdd(counts + 1, (unsigned long long)nsec);
      atomicAdd(counts + 2, (unsigned long long)nrec);
    }
  }
}

constexpr int kLookupThreads = 256;

// Host-buffer lookup: keys read and results written in place in pinned host
// memory over NVLink-C2C. Small scattered stores are what the link does worst,
// so a block stages its 256 values and 256 flags in shared memory and writes
// them out as 16-byte vectors (2 KB + 256 B per block); keys come in as one
// coalesced 16-byte load per thread.
template <bool kTimers>
__global__ void __launch_bounds__(kLookupThreads) lookup_host_kernel(TableView t, const uint8_t* __restrict__ keys,
                                                                     uint64_t n, uint64_t* __restrict__ out_vals,
                                                                     uint8_t* __restrict__ out_found, uint32_t now,
                                                                     uint32_t refresh_ttl) {
  __shared__ __align__(16) uint64_t vals[kLookupThreads];
  __shared__ __align__(16) uint8_t flags[kLookupThreads];
  const uint64_t base = (uint64_t)blockIdx.x * kLookupThreads;
  const uint64_t i = base + threadIdx.x;
  uint64_t value = 0;
  bool found = false;
  if (i < n) {
    const uint64_t keep = policy_evict_last();
    const uint64_t stream = policy_evict_first();
    const ulonglong2 kk = *reinterpret_cast<const ulonglong2*>(keys + 16 * i);
    uint32_t nsec = 0, nrec = 0;
    found = probe_key<kTimers, false, kBloom>(t, Key{kk.x, kk.y}, now, refresh_ttl, keep, stream, value, nsec, nrec);
  }
  vals[threadIdx.x] = value;
  flags[threadIdx.x] = found ? 1 : 0;
  __syncthreads();
  if (base + kLookupThreads <= n) {
    // full block: 128 threads store the values, 16 the flags, 16 bytes each
    if (threadIdx.x < kLookupThreads / 2) {
      reinterpret_cast<ulonglong2*>(out_vals + base)[threadIdx.x] =
          reinterpret_cast<const ulonglong2*>(vals)[threadIdx.x];
    } else if (threadIdx.x < kLookupThreads / 2 + kLookupThreads / 16) {
      const int j = threadIdx.x - kLookupThreads / 2;
      reinterpret_cast<uint4*>(out_found + base)[j] = reinterpret_cast<const uint4*>(flags)[j];
    }
  } else if (i < n) {
    out_vals[i] = vals[threadIdx.x];
    out_found[i] = flags[threadIdx.x];
  }
}

template <bool kTimers, bool kCount, bool kHostIO, int kVariant>
cudaError_t launch(const TableView& t, const uint8_t* keys, uint64_t n, uint64_t* out_vals, uint8_t* out_found,
                   uint32_t now, uint32_t refresh_ttl, unsigned long long* counts, cudaStream_t s) {
  const uint64_t blocks = (n + kLookupThreads - 1) / kLookupThreads;
  lookup_kernel<kTimers, kCount, kHostIO, kVariant><<<(unsigned)blocks, kLookupThreads, 0, s>>>(
      t, keys, n, out_vals, out_found, now, refresh_ttl, counts);
  return cudaGetLastError();
}

template <bool kCount, int kVariant>
cudaError_t launch_variant(const TableView& t, const uint8_t* keys, uint64_t n, uint64_t* out_vals,
                           uint8_t* out_found, uint32_t now, uint32_t refresh_ttl, unsigned long long* counts,
                           cudaStream_t s) {
  if (t.timers) return launch<true, kCount, false, kVariant>(t, keys, n, out_vals, out_found, now, refresh_ttl, counts, s);
  return launch<false, kCount, false, kVariant>(t, keys, n, out_vals, out_found, now, 0, counts, s);
}

}  // namespace

cudaError_t launch_lookup(const TableView& t, const uint8_t* keys, uint64_t n, uint64_t* out_vals,
                          uint8_t* out_found, uint32_t now, uint32_t refresh_ttl, bool host_io, int variant,
                          cudaStream_t s) {
  if (host_io) {
    if (variant != kBloom) return cudaErrorInvalidValue;
    const bool vec = (reinterpret_cast<uintptr_t>(out_vals) % 16 == 0) && (reinterpret_cast<uintptr_t>(out_found) % 16 == 0);
    if (vec) {
      const unsigned blocks = (unsigned)((n + kLookupThreads - 1) / kLookupThreads);
      if (t.timers) {
        lookup_host_kernel<true><<<blocks, kLookupThreads, 0, s>>>(t, keys, n, out_vals, out_found, now, refresh_ttl);
      } else {
        lookup_host_kernel<false><<<blocks, kLookupThreads, 0, s>>>(t, keys, n, out_vals, out_found, now, 0);
      }
      return cudaGetLastError();
    }
    if (t.timers) return launch<true, false, true, kBloom>(t, keys, n, out_vals, out_found, now, refresh_ttl, nullptr, s);
    return launch<false, false, true, kBloom>(t, keys, n, out_vals, out_found, now, 0, nullptr, s);
  }
  switch (variant) {
    case kBloom: return launch_variant<false, kBloom>(t, keys, n, out_vals, out_found, now, refresh_ttl, nullptr, s);
    case kOptimistic:
      return launch_variant<false, kOptimistic>(t, keys, n, out_vals, out_found, now, refresh_ttl, nullptr, s);
    case kPessimistic:
      return launch_variant<false, kPessimistic>(t, keys, n, out_vals, out_found, now, refresh_ttl, nullptr, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_probe_counts(const TableView& t, const uint8_t* keys, uint64_t n, uint32_t now, int variant,
                                unsigned long long* counts, cudaStream_t s) {
  switch (variant) {
    case kBloom: return launch_variant<true, kBloom>(t, keys, n, nullptr, nullptr, now, 0, counts, s);
    case kOptimistic: return launch_variant<true, kOptimistic>(t, keys, n, nullptr, nullptr, now, 0, counts, s);
    case kPessimistic: return launch_variant<true, kPessimistic>(t, keys, n, nullptr, nullptr, now, 0, counts, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ckpp
