// Bulk lookup over one table (Sec. 2 and Sec. 4.1 of the paper): each warp
// takes 32 keys, one per lane, and fetches their bucket lines together into
// shared memory (probe.cuh).
//
// The paper hides DRAM latency by interleaving the steps of a batch of lookups
// with prefetches (Sec. 3); on the GPU the same memory-level parallelism comes
// from every warp keeping its 32 keys' line requests in flight at once, over
// the tens of warps resident on each SM. Blocks are short-lived and launched in
// key order, so at any time the resident warps read keys, and write results,
// within one narrow window of the batch. (Measured: warps that each walk a long
// span of the batch, with their next keys prefetched, ran 10-20% slower.)
// Keys are read with coalesced 16-byte loads and results written with
// coalesced stores.
#include "probe.cuh"

namespace ckpp {

namespace {

constexpr int kLookupThreads = 128;  // 4 warps: 17 KB of line slabs per block
constexpr int kWarpsPerBlock = kLookupThreads / 32;

// kHostIO: keys and results live in pinned host memory, reached over
// NVLink-C2C by the loads and stores themselves (no staging copy); such keys
// are read with plain loads, without the read-only path or L2 hints, and each
// warp writes its results as 16-byte vectors (small scattered stores are what
// the link does worst) when the output pointers allow it.
// kCount: no results; the secondary-line, record and second-line reads are
// added to counts[1..3] and the keys to counts[0].
template <bool kCount, bool kHostIO, int kVariant, int kTM>
__global__ void __launch_bounds__(kLookupThreads) lookup_kernel(TableView t, const uint8_t* __restrict__ keys,
                                                                uint64_t n, uint64_t* __restrict__ out_vals,
                                                                uint8_t* __restrict__ out_found, uint32_t now,
                                                                uint32_t refresh_ttl,
                                                                unsigned long long* __restrict__ counts) {
  __shared__ WarpStage<1> stage[kWarpsPerBlock];
  __shared__ __align__(16) uint64_t vals[kHostIO ? kLookupThreads : 1];
  __shared__ __align__(16) uint8_t flags[kHostIO ? kLookupThreads : 1];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t c = (uint64_t)blockIdx.x * kWarpsPerBlock + warp;  // the warp's 32-key chunk
  const uint64_t i = c * 32 + lane;
  bool act[1] = {i < n};
  Key k{0, 0};
  if (act[0]) {
    if (kHostIO) {
      const ulonglong2 kk = *reinterpret_cast<const ulonglong2*>(keys + 16 * i);
      k = Key{kk.x, kk.y};
    } else {
      k = ld_key_ro(keys + 16 * i, policy_evict_first());
    }
  }
  Probe p[1];
  probe_init(p[0], k, t.buckets, t.nb, t.seed, t.timers);
  run_probes<kVariant, kCount, 1, kTM>(p, act, now, stage[warp]);
  if (kCount) {
    const uint32_t nkey = __reduce_add_sync(kFull, act[0] ? 1u : 0u);
    const uint32_t nsec = __reduce_add_sync(kFull, p[0].nsec);
    const uint32_t nrec = __reduce_add_sync(kFull, p[0].nrec);
    const uint32_t nl1 = __reduce_add_sync(kFull, p[0].nline1);
    if (lane == 0 && nkey) {
      atomicAdd(counts + 0, (unsigned long long)nkey);
      atomicAdd(counts + 1, (unsigned long long)nsec);
      atomicAdd(counts + 2, (unsigned long long)nrec);
      atomicAdd(counts + 3, (unsigned long long)nl1);
    }
    return;
  }
  // Sec. 4.2: a hit may refresh the entry's expiry.
  if (kTM == kWithTimers && act[0] && p[0].found && refresh_ttl) set_expiry(t, p[0].hb, p[0].hs, now + refresh_ttl);
  const bool vec = kHostIO && (reinterpret_cast<uintptr_t>(out_vals) % 16 == 0) &&
                   (reinterpret_cast<uintptr_t>(out_found) % 16 == 0);
  if (vec && c * 32 + 32 <= n) {
    uint64_t* wv = vals + warp * 32;
    uint8_t* wf = flags + warp * 32;
    wv[lane] = p[0].value;
    wf[lane] = p[0].found ? 1 : 0;
    __syncwarp();
    if (lane < 16) {
      reinterpret_cast<ulonglong2*>(out_vals + c * 32)[lane] = reinterpret_cast<const ulonglong2*>(wv)[lane];
    } else if (lane < 18) {
      reinterpret_cast<uint4*>(out_found + c * 32)[lane - 16] = reinterpret_cast<const uint4*>(wf)[lane - 16];
    }
  } else if (act[0]) {
    out_vals[i] = p[0].value;
    out_found[i] = p[0].found ? 1 : 0;
  }
}

template <bool kCount, bool kHostIO, int kVariant>
cudaError_t launch(const TableView& t, const uint8_t* keys, uint64_t n, uint64_t* out_vals, uint8_t* out_found,
                   uint32_t now, uint32_t refresh_ttl, unsigned long long* counts, cudaStream_t s) {
  const uint64_t blocks = ((n + 31) / 32 + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (t.timers) {
    lookup_kernel<kCount, kHostIO, kVariant, kWithTimers><<<(unsigned)blocks, kLookupThreads, 0, s>>>(
        t, keys, n, out_vals, out_found, now, refresh_ttl, counts);
  } else {
    lookup_kernel<kCount, kHostIO, kVariant, kNoTimers><<<(unsigned)blocks, kLookupThreads, 0, s>>>(
        t, keys, n, out_vals, out_found, now, 0u, counts);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_lookup(const TableView& t, const uint8_t* keys, uint64_t n, uint64_t* out_vals,
                          uint8_t* out_found, uint32_t now, uint32_t refresh_ttl, bool host_io, int variant,
                          cudaStream_t s) {
  if (host_io) {
    if (variant != kBloom) return cudaErrorInvalidValue;
    return launch<false, true, kBloom>(t, keys, n, out_vals, out_found, now, refresh_ttl, nullptr, s);
  }
  switch (variant) {
    case kBloom: return launch<false, false, kBloom>(t, keys, n, out_vals, out_found, now, refresh_ttl, nullptr, s);
    case kOptimistic:
      return launch<false, false, kOptimistic>(t, keys, n, out_vals, out_found, now, refresh_ttl, nullptr, s);
    case kPessimistic:
      return launch<false, false, kPessimistic>(t, keys, n, out_vals, out_found, now, refresh_ttl, nullptr, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_probe_counts(const TableView& t, const uint8_t* keys, uint64_t n, uint32_t now, int variant,
                                unsigned long long* counts, cudaStream_t s) {
  switch (variant) {
    case kBloom: return launch<true, false, kBloom>(t, keys, n, nullptr, nullptr, now, 0, counts, s);
    case kOptimistic: return launch<true, false, kOptimistic>(t, keys, n, nullptr, nullptr, now, 0, counts, s);
    case kPessimistic: return launch<true, false, kPessimistic>(t, keys, n, nullptr, nullptr, now, 0, counts, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ckpp
