// The per-key lookup of the method, shared by the plain, counting and batched
// lookup kernels (Sec. 2 and Sec. 4.1 of the paper, Fig. 4).
//
// Per key: two hashes in registers, one 32-byte read of the primary bucket's
// hot sector (tags, Bloom filter, busy mask), one 32-byte key/value record read
// per tag match, and -- after a primary miss -- the secondary bucket.
//
// Which secondary reads happen is the lookup strategy:
//   kBloom        Cuckoo++ (Sec. 4.1): only if both filter bits of the
//                 primary are set;
//   kOptimistic   the optimistic strategy of Sec. 3: on every primary miss;
//   kPessimistic  the pessimistic strategy of Sec. 3: the secondary bucket is
//                 read together with the primary for every key.
// All three return identical results; they differ only in memory reads, which
// is what the ablation measures.
#pragma once

#include "ckpp_kernels.h"

namespace ckpp {

enum LookupVariant : int { kBloom = 0, kOptimistic = 1, kPessimistic = 2 };

// Confirm the candidate slots of bucket b (tag matches among busy slots) by
// reading their records. Returns the matching slot or -1; rec holds its record.
// With timers the record carries a copy of the slot's 16-bit expiry (its low
// bytes 24..25), so the alive test costs no read beyond the record itself.
template <bool kTimers, bool kCount>
__device__ __forceinline__ int confirm(const TableView& t, uint32_t b, uint32_t cand, const Key& k, uint64_t pol,
                                       uint64_t (&rec)[4], uint32_t& expiry, uint32_t& nrec) {
  while (cand) {
    const int s = __ffs(cand) - 1;
    cand &= cand - 1;
    ld256_ro(record_ptr(t, b, s), pol, rec);
    if (kTimers) expiry = (uint32_t)(rec[3] & 0xFFFFu);
    if (kCount) ++nrec;
    if (same_key(rec, k)) return s;
  }
  return -1;
}

__device__ __forceinline__ uint32_t candidates(const uint64_t (&h)[4], uint32_t tag) {
  return tag_mask(h[0], h[1], tag) & (uint32_t)h[3] & kBusyMask;
}

// Look key k up in table t. Returns found; value receives the value (0 on a
// miss). keep / stream are the L2 policies for bucket and record reads. With
// kCount the secondary-bucket and record reads are added to nsec / nrec and
// no expiry is refreshed.
template <bool kTimers, bool kCount, int kVariant>
__device__ __forceinline__ bool probe_key(const TableView& t, const Key& k, uint32_t now, uint32_t refresh_ttl,
                                          uint64_t keep, uint64_t stream, uint64_t& value, uint32_t& nsec,
                                          uint32_t& nrec) {
  const Addr a = address_of(k, t.nb, t.seed);
  uint64_t h[4], h2[4], rec[4];
  uint32_t expiry = 0;
  ld256_ro(bucket_ptr(t, a.b1), keep, h);
  if (kVariant == kPessimistic) {
    ld256_ro(bucket_ptr(t, a.b2), keep, h2);
    if (kCount) ++nsec;
  }
  uint32_t b = a.b1;
  int s = confirm<kTimers, kCount>(t, b, candidates(h, a.tag), k, stream, rec, expiry, nrec);
  if (s < 0) {
    const bool read2 = kVariant == kBloom ? (h[2] & a.bits) == a.bits : true;
    if (read2) {
      if (kVariant != kPessimistic) {
        ld256_ro(bucket_ptr(t, a.b2), keep, h2);
        if (kCount) ++nsec;
      }
      b = a.b2;
      s = confirm<kTimers, kCount>(t, b, candidates(h2, a.tag), k, stream, rec, expiry, nrec);
    }
  }
  bool found = s >= 0;
  // Sec. 4.2: a dead entry is ignored; a hit may refresh the expiry.
  if (kTimers && found) {
    found = alive16(expiry, now);
    if (!kCount && found && refresh_ttl) set_expiry(t, b, s, now + refresh_ttl);
  }
  value = found ? rec[2] : 0ull;
  return found;
}

}  // namespace ckpp
