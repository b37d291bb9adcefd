// Device helpers shared by the mutating kernels (insert, delete, expire):
// bucket locks, bucket snapshots, slot placement and removal with the moved
// counter and Bloom filter upkeep of Sec. 4.1.
//
// Concurrency rules of the insert kernels (one table, one batch at a time):
//  * phase 1 takes no lock: a key claims a free or dead slot with a CAS on the
//    bucket's ctrl word (claimed bits 16-23), writes its entry into the
//    claimed slot, and the next kernel publishes the claim (claimed -> busy);
//    searches look at busy slots only, so a claimed slot is invisible until
//    then. In-place updates touch live entries, which no claim can take;
//  * in the displacement passes (after publication) a bucket's busy /
//    in_secondary bits, tags, expiries, keys and values change only while its
//    lock bit (ctrl bit 31) is held; the new ctrl word is published by the
//    unlocking exchange;
//  * Bloom bits of bucket p are set in phase 1 (no reset runs there) or under
//    p's lock, and a filter is reset only under p's lock or after the batch,
//    so a reset cannot erase a concurrent insertion's bits;
//  * a moved counter may be decremented without its bucket's lock (when a dead
//    entry is overwritten elsewhere); a decrement that reaches zero off-lock
//    queues the bucket for a reset pass that runs after the batch.
// Every wait is bounded: a lock not taken after kLockSpins tries (or a claim
// whose CAS keeps failing) gives up; the caller reports CKPP_ST_BUSY and
// latches kErrLockTimeout.
#pragma once

#include "ckpp_kernels.h"

namespace ckpp {

// The kernels of one insert or delete call run back to back on one stream,
// each launched with programmatic stream serialization, so that the GPU can
// schedule a kernel while its predecessor finishes instead of after it.
// Each such kernel calls pdl_wait() before touching memory: it returns once
// the predecessor grid has completed and its writes are visible (for a kernel
// launched without the attribute it returns at once). pdl_release() lets the
// successor be scheduled; it does not let the successor past its own wait.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Lock word access: taking a lock is an acquire (later reads see what the
// previous holder wrote), releasing it a release (everything written under the
// lock is visible before the word clears). No full fence is needed.
__device__ __forceinline__ uint32_t or_acquire(uint32_t* p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.acquire.gpu.global.or.b32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ void exch_release(uint32_t* p, uint32_t v) {
  [[maybe_unused]] uint32_t old;
  asm volatile("atom.release.gpu.global.exch.b32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
}

// Relaxed forms for several lock words at once: the atomics of a group are
// issued together, and one fence gives the group acquire (after) or release
// (before) ordering.
__device__ __forceinline__ uint32_t or_relaxed(uint32_t* p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.relaxed.gpu.global.or.b32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ void and_relaxed(uint32_t* p, uint32_t v) {
  [[maybe_unused]] uint32_t old;
  asm volatile("atom.relaxed.gpu.global.and.b32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void exch_relaxed(uint32_t* p, uint32_t v) {
  [[maybe_unused]] uint32_t old;
  asm volatile("atom.relaxed.gpu.global.exch.b32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// A bucket lock is held for microseconds (one cuckoo path's moves); a waiter
// gives up after about 0.2 s of polls with back-off (each poll an atomic and a
// sleep of up to 1 us), far longer than any holder, and well inside the grid
// barrier's bound of the single-launch insert.
constexpr int kLockSpins = 1 << 17;

__device__ __forceinline__ bool lock_bucket(const TableView& t, uint32_t b, uint32_t& ctrl) {
  uint32_t* c = ctrl_ptr(t, b);
  for (int i = 0; i < kLockSpins; ++i) {
    const uint32_t old = or_acquire(c, kLockBit);
    if (!(old & kLockBit)) {
      ctrl = old;
      return true;
    }
    __nanosleep(32u << (i < 5 ? i : 5));
  }
  return false;
}

__device__ __forceinline__ void unlock_bucket(const TableView& t, uint32_t b, uint32_t ctrl) {
  exch_release(ctrl_ptr(t, b), ctrl & ~kLockBit);
}

// Lock the n buckets b[0..n) (ascending, distinct), returning their words in
// ctrl. First all lock bits are set at once; if any was held, the ones taken
// are dropped again and the buckets are locked one by one in index order (a
// global order, so waiters cannot deadlock). False if a wait gave up (nothing
// is then held).
template <int N>
__device__ __forceinline__ bool lock_buckets(const TableView& t, const uint32_t (&b)[N], int n, uint32_t (&ctrl)[N]) {
  bool all = true;
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (i < n) ctrl[i] = or_relaxed(ctrl_ptr(t, b[i]), kLockBit);
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (i < n) all &= !(ctrl[i] & kLockBit);
  if (all) {
    fence_acq_rel();  // acquire: the holders' writes before their release are seen from here on
    return true;
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (i < n && !(ctrl[i] & kLockBit)) and_relaxed(ctrl_ptr(t, b[i]), ~kLockBit);  // nothing written: drop it
  for (int i = 0; i < n; ++i) {
    if (!lock_bucket(t, b[i], ctrl[i])) {
      for (int j = i - 1; j >= 0; --j) unlock_bucket(t, b[j], ctrl[j]);
      return false;
    }
  }
  return true;
}

// Store the words ctrl[0..n) (lock bits cleared) into the locked buckets b,
// after one release fence for all of them.
template <int N>
__device__ __forceinline__ void unlock_buckets(const TableView& t, const uint32_t (&b)[N], int n,
                                               const uint32_t (&ctrl)[N]) {
  fence_acq_rel();
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (i < n) exch_relaxed(ctrl_ptr(t, b[i]), ctrl[i] & ~kLockBit);
}

// The bucket an entry of bucket x can move to, from one hash of its key e: its
// primary if it lives in its secondary (in_secondary bit set), else its
// secondary (Sec. 2; the same collapse rule as address_of when the two hashes
// pick the same bucket). The bit selects the hash's seed, so lanes of a warp
// with different bits run the same instructions.
__device__ __forceinline__ uint32_t other_bucket(const Key& e, uint32_t x, bool insec, uint64_t nb, uint64_t seed) {
  const uint32_t o = reduce(hash_key(e, insec ? seed : seed ^ kSeed2Xor), nb);
  const uint32_t next = x + 1 == (uint32_t)nb ? 0u : x + 1;
  return (!insec && o == x) ? next : o;
}

// The control word and the 8 keys of bucket b, read one 32-byte sector per
// request: the keys of two slots share a sector, so the 8 keys and the word
// take 5 requests (6 with timers) instead of 9 (bucket layout in
// ckpp_device.cuh).
__device__ __forceinline__ uint32_t load_bucket_keys(const TableView& t, uint32_t b, uint64_t (&k0)[kSlots],
                                                     uint64_t (&k1)[kSlots]) {
  const uint8_t* p = bucket_ptr(t, b);
  uint64_t h[4], s1[4], s2[4], s3[4], s4[4], s5[4] = {0, 0, 0, 0};
  ld256_cg(p, h);
  ld256_cg(p + 32, s1);
  ld256_cg(p + 64, s2);
  ld256_cg(p + 128, s3);
  ld256_cg(p + 160, s4);
  if (t.timers) ld256_cg(p + 192, s5);
  if (!t.timers) {  // keys 0..3 at bytes 32..95, keys 4..7 at 128..191
    k0[0] = s1[0], k1[0] = s1[1], k0[1] = s1[2], k1[1] = s1[3];
    k0[2] = s2[0], k1[2] = s2[1], k0[3] = s2[2], k1[3] = s2[3];
    k0[4] = s3[0], k1[4] = s3[1], k0[5] = s3[2], k1[5] = s3[3];
    k0[6] = s4[0], k1[6] = s4[1], k0[7] = s4[2], k1[7] = s4[3];
  } else {  // keys 0..2 at bytes 48..95, keys 3..7 at 128..207
    k0[0] = s1[2], k1[0] = s1[3];
    k0[1] = s2[0], k1[1] = s2[1], k0[2] = s2[2], k1[2] = s2[3];
    k0[3] = s3[0], k1[3] = s3[1], k0[4] = s3[2], k1[4] = s3[3];
    k0[5] = s4[0], k1[5] = s4[1], k0[6] = s4[2], k1[6] = s4[3];
    k0[7] = s5[0], k1[7] = s5[1];
  }
  return (uint32_t)h[3];  // ctrl: bytes 24..27
}

// Coherent snapshot of a bucket: its first sector and (with timers) the 8 expiries.
struct Snap {
  uint64_t w[4];
  uint64_t e0, e1;
};

__device__ __forceinline__ void snap_bucket(const TableView& t, uint32_t b, Snap& s) {
  ld256_cg(bucket_ptr(t, b), s.w);
  if (t.timers) {
    ld128_cg(expiry_ptr(t, b, 0), s.e0, s.e1);
  } else {
    s.e0 = s.e1 = 0;
  }
}

__device__ __forceinline__ uint32_t snap_expiry(const Snap& s, uint32_t slot) {
  const uint64_t e = slot < 4 ? s.e0 : s.e1;
  return (uint32_t)(e >> (16 * (slot & 3))) & 0xFFFFu;
}

// Slots an insertion may take: empty, or busy with a dead entry (Sec. 4.2).
__device__ __forceinline__ uint32_t free_mask(const TableView& t, uint32_t ctrl, const Snap& s, uint32_t now) {
  const uint32_t busy = ctrl & kBusyMask;
  uint32_t f = ~busy & kBusyMask;
  if (t.timers) f |= busy & ~alive_mask(s.e0, s.e1, now) & kBusyMask;
  return f;
}

// Slot of bucket b holding key k (alive or dead), or -1.
__device__ __forceinline__ int find_key(const TableView& t, uint32_t b, uint32_t ctrl, const Snap& s, const Key& k,
                                        uint32_t tag) {
  uint32_t cand = tag_mask(s.w[0], s.w[1], tag) & ctrl & kBusyMask;
  while (cand) {
    const int slot = __ffs(cand) - 1;
    cand &= cand - 1;
    uint64_t k0, k1;
    ld128_cg(key_ptr(t, b, slot), k0, k1);
    if (k0 == k.k0 && k1 == k.k1) return slot;
  }
  return -1;
}

__device__ __forceinline__ void push_fixup(const Workspace& ws, uint32_t table, uint32_t b) {
  const uint32_t idx = atomicAdd(ws.counters + 1, 1u);
  if (idx < ws.fix_cap) {
    ws.fixup[idx] = ((unsigned long long)table << 32) | b;
  } else {
    atomicExch(ws.counters + 2, 1u);
  }
}

// Remove the (dead) entry in slot s of locked bucket b of table tid: if it sits in its
// secondary bucket its primary's moved counter is decremented (Sec. 4.1).
__device__ __forceinline__ void evict_entry(const TableView& t, uint32_t tid, uint32_t b, uint32_t s, uint32_t& ctrl,
                                            const Workspace& ws) {
  if ((ctrl >> (kInsecShift + s)) & 1u) {
    Key k;
    ld128_cg(key_ptr(t, b, s), k.k0, k.k1);
    const Addr a = address_of(k, t.nb, t.seed);
    const uint32_t old = atomicSub(moved_ptr(t, a.b1), 1u);
    if (old == 1u) push_fixup(ws, tid, a.b1);
  }
  ctrl &= ~((1u << s) | (1u << (kInsecShift + s)));
}

// Store a new entry in free slot s of locked bucket b; if b is the key's
// secondary bucket, set its two bits in the primary's filter and increment the
// primary's moved counter (Sec. 4.1). The caller holds the primary's lock too.
__device__ __forceinline__ void place_entry(const TableView& t, uint32_t b, uint32_t s, const Key& k, uint64_t v,
                                            const Addr& a, uint32_t expiry, uint32_t& ctrl) {
  st128_cg(key_ptr(t, b, s), k.k0, k.k1);
  st64_cg(value_ptr(t, b, s), v);
  st16_cg(tag_ptr(t, b, s), a.tag);
  if (t.timers) st16_cg(expiry_ptr(t, b, s), expiry);
  ctrl |= 1u << s;
  if (b == a.b2) {
    ctrl |= 1u << (kInsecShift + s);
    atomicOr(reinterpret_cast<unsigned long long*>(bloom_ptr(t, a.b1)), (unsigned long long)a.bits);
    atomicAdd(moved_ptr(t, a.b1), 1u);
  } else {
    ctrl &= ~(1u << (kInsecShift + s));
  }
}

}  // namespace ckpp
