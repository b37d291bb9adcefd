// Batched lookup (Sec. 2 and Sec. 4.1 of the paper, Fig. 4): one thread per key.
//
// Per key: a coalesced 16-byte key load, two hashes in registers, one 32-byte
// read of the primary bucket's hot sector (tags, Bloom filter, busy mask), a
// 32-byte key/value record read per tag match, and -- only after a primary miss
// whose two Bloom bits are both set -- the same on the secondary bucket.
// Negative lookups therefore touch one random sector in almost all cases, and
// positive lookups two (three when the key lives in its secondary bucket).
//
// The paper hides DRAM latency by interleaving the steps of a batch of lookups
// with prefetches (Sec. 3); on the GPU the same memory-level parallelism comes
// from tens of thousands of resident threads, each with its own chain of loads.
#include "ckpp_kernels.h"

namespace ckpp {

namespace {

// Confirm the candidate slots of bucket b (tag matches among busy slots) by
// reading their records. Returns the matching slot or -1; rec holds its record.
// With timers the candidate's expiry is fetched alongside its record.
template <bool kTimers, bool kCount>
__device__ __forceinline__ int confirm(const TableView& t, uint32_t b, uint32_t cand, const Key& k, uint64_t pol,
                                       uint64_t (&rec)[4], uint32_t& expiry, uint32_t& nrec) {
  while (cand) {
    const int s = __ffs(cand) - 1;
    cand &= cand - 1;
    if (kTimers) expiry = ld16_cg(expiry_ptr(t, b, s));
    ld256_ro(record_ptr(t, b, s), pol, rec);
    if (kCount) ++nrec;
    if (same_key(rec, k)) return s;
  }
  return -1;
}

// kHostIO: keys and results live in pinned host memory, reached over
// NVLink-C2C by the loads and stores themselves (no staging copy); such keys
// are read with plain loads, without the read-only path or L2 hints.
template <bool kTimers, bool kCount, bool kHostIO>
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
    const Addr a = address_of(k, t.nb, t.seed);
    uint64_t h[4], rec[4];
    uint32_t expiry = 0;
    ld256_ro(bucket_ptr(t, a.b1), keep, h);
    uint32_t b = a.b1;
    int s = confirm<kTimers, kCount>(t, b, tag_mask(h[0], h[1], a.tag) & (uint32_t)h[3] & kBusyMask, k, stream, rec,
                                     expiry, nrec);
    // Sec. 4.1: the secondary bucket is read only if both filter bits are set.
    if (s < 0 && (h[2] & a.bits) == a.bits) {
      if (kCount) ++nsec;
      b = a.b2;
      ld256_ro(bucket_ptr(t, b), keep, h);
      s = confirm<kTimers, kCount>(t, b, tag_mask(h[0], h[1], a.tag) & (uint32_t)h[3] & kBusyMask, k, stream, rec,
                                   expiry, nrec);
    }
    bool found = s >= 0;
    // Sec. 4.2: a dead entry is ignored; a hit may refresh the expiry.
    if (kTimers && found) {
      found = alive16(expiry, now);
      if (!kCount && found && refresh_ttl) st16_cg(expiry_ptr(t, b, s), now + refresh_ttl);
    }
    if (kCount) {
      nkey = 1;
    } else {
      out_vals[i] = found ? rec[2] : 0ull;
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

template <bool kTimers, bool kCount, bool kHostIO = false>
cudaError_t launch(const TableView& t, const uint8_t* keys, uint64_t n, uint64_t* out_vals, uint8_t* out_found,
                   uint32_t now, uint32_t refresh_ttl, unsigned long long* counts, cudaStream_t s) {
  const uint64_t blocks = (n + kLookupThreads - 1) / kLookupThreads;
  lookup_kernel<kTimers, kCount, kHostIO><<<(unsigned)blocks, kLookupThreads, 0, s>>>(
      t, keys, n, out_vals, out_found, now, refresh_ttl, counts);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_lookup(const TableView& t, const uint8_t* keys, uint64_t n, uint64_t* out_vals,
                          uint8_t* out_found, uint32_t now, uint32_t refresh_ttl, bool host_io, cudaStream_t s) {
  if (host_io) {
    if (t.timers) return launch<true, false, true>(t, keys, n, out_vals, out_found, now, refresh_ttl, nullptr, s);
    return launch<false, false, true>(t, keys, n, out_vals, out_found, now, 0, nullptr, s);
  }
  if (t.timers) return launch<true, false>(t, keys, n, out_vals, out_found, now, refresh_ttl, nullptr, s);
  return launch<false, false>(t, keys, n, out_vals, out_found, now, 0, nullptr, s);
}

cudaError_t launch_probe_counts(const TableView& t, const uint8_t* keys, uint64_t n, uint32_t now,
                                unsigned long long* counts, cudaStream_t s) {
  if (t.timers) return launch<true, true>(t, keys, n, nullptr, nullptr, now, 0, counts, s);
  return launch<false, true>(t, keys, n, nullptr, nullptr, now, 0, counts, s);
}

}  // namespace ckpp
