// The per-key lookup of the method (Sec. 2 and Sec. 4.1 of the paper, Fig. 4),
// run over the 256-byte bucket layout of ckpp_device.cuh.
//
// Per key: two hashes; the primary bucket's first line (tags, filter, busy
// mask and the entries of the first slots); its second line only if a tag of
// the other slots matches; after a primary miss, the secondary bucket in the
// same way.
//
// How a line is read: a random access costs one 128-byte line request whether
// it brings 32 bytes or the whole line, but only if the line's sectors are
// requested by one warp instruction; a thread's second read of the same line
// costs a second access. So each key's owner lane posts the address of the
// line it needs next; the warp copies all posted lines into its shared-memory
// slab with cp.async (8 lanes x 16 bytes per line, four lines per instruction);
// then each owner examines its own line there with plain per-thread code and
// either finishes or posts its next line. Lines are fetched for every key of
// the warp at once, so a warp keeps up to 32 x G line requests in flight.
//
// Which secondary reads happen is the lookup strategy:
//   kBloom        Cuckoo++ (Sec. 4.1): only if both filter bits of the
//                 primary are set;
//   kOptimistic   the optimistic strategy of Sec. 3: on every primary miss;
//   kPessimistic  the pessimistic strategy of Sec. 3: the secondary bucket's
//                 first line is read for every key, also after a primary hit.
// All three return identical results; they differ only in memory reads, which
// is what the ablation measures.
#pragma once

#include "ckpp_kernels.h"

namespace ckpp {

enum LookupVariant : int { kBloom = 0, kOptimistic = 1, kPessimistic = 2 };

constexpr uint32_t kFull = 0xFFFFFFFFu;

// Whether the keys' tables have timers: known for the whole launch (a plain
// lookup is over one table) or per key (the batched form).
enum TimersMode : int { kNoTimers = 0, kWithTimers = 1, kTimersPerKey = 2 };
constexpr uint32_t kDone = 4;  // stages: 0 b1 line 0, 1 b1 line 1, 2 b2 line 0, 3 b2 line 1, 4 done

// One key's lookup, owned by one lane.
struct Probe {
  Key k;
  const uint8_t* buckets;  // the key's table
  uint32_t b1, b2, tag;
  uint32_t bidx;    // the two filter bit indices: i1 | i2 << 6
  uint32_t timers;  // the table has timers
  uint32_t stage;
  uint32_t carry;   // for a second-line job: its tag-matching slots | alive mask << 8
  bool bloom_ok;    // both filter bits of the primary are set
  bool skip;        // pessimistic: the key is resolved; the read is made for its cost only
  bool found;
  uint64_t value;
  uint32_t hb, hs;  // bucket and slot of the hit (for a refresh)
  uint32_t nsec, nrec, nline1;  // counting mode
};

__device__ __forceinline__ void probe_init(Probe& p, const Key& k, const uint8_t* buckets, uint64_t nb, uint64_t seed,
                                           uint32_t timers) {
  const uint64_t h1 = hash_key(k, seed);
  const uint64_t h2 = hash_key(k, seed ^ kSeed2Xor);
  p.k = k;
  p.buckets = buckets;
  p.b1 = reduce(h1, nb);
  p.b2 = reduce(h2, nb);
  if (p.b2 == p.b1) p.b2 = (p.b1 + 1 == (uint32_t)nb) ? 0u : p.b1 + 1;
  p.tag = (uint32_t)(h1 & 0xFFFF);
  p.bidx = (uint32_t)(h2 & 63) | (uint32_t)((h2 >> 6) & 63) << 6;
  p.timers = timers;
  p.stage = 0;
  p.carry = 0;
  p.bloom_ok = false;
  p.skip = false;
  p.found = false;
  p.value = 0;
  p.hb = p.hs = 0;
  p.nsec = p.nrec = p.nline1 = 0;
}

// Shared-memory slab of one warp: the line jobs of an iteration, posted by
// their owners at their rank, and the lines themselves. Line j's 16-byte
// chunk c is stored at chunk c ^ (j & 7), so the owners of lines 0..7 reading
// the same field hit eight different bank groups.
template <int G>
struct WarpStage {
  unsigned long long addr[32 * G];
  __align__(128) uint8_t line[32 * G][kLineBytes];
};

__device__ __forceinline__ uint4 lds128(const uint8_t* p) { return *reinterpret_cast<const uint4*>(p); }
__device__ __forceinline__ uint64_t lds64(const uint8_t* p) { return *reinterpret_cast<const uint64_t*>(p); }
__device__ __forceinline__ uint64_t lo64(const uint4& v) { return (uint64_t)v.x | (uint64_t)v.y << 32; }
__device__ __forceinline__ uint64_t hi64(const uint4& v) { return (uint64_t)v.z | (uint64_t)v.w << 32; }

// Mask of the 8 tags (16-bit lanes of tg) equal to tag: per 32-bit word, a
// 16-bit lane of x = word ^ (tag, tag) is zero exactly when the top bit of
// ((x & 0x7FFF) + 0x7FFF) | x is clear, with no carry between lanes.
__device__ __forceinline__ uint32_t tag_mask16(const uint4& tg, uint32_t tag) {
  const uint32_t rep = tag * 0x00010001u;
  const uint32_t w[4] = {tg.x ^ rep, tg.y ^ rep, tg.z ^ rep, tg.w ^ rep};
  uint32_t q = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t z = ~(((w[i] & 0x7FFF7FFFu) + 0x7FFF7FFFu) | w[i]) & 0x80008000u;  // bit 15 / 31: lane is zero
    q |= z >> (15 - 2 * i);  // slot 2i -> bit 2i, slot 2i+1 -> bit 2i+16
  }
  return (q & 0x55u) | ((q >> 15) & 0xAAu);
}

template <int kVariant>
__device__ __forceinline__ void resolve(Probe& p, bool found, uint64_t value, uint32_t b, uint32_t slot) {
  p.found = found;
  p.value = found ? value : 0ull;
  p.hb = b;
  p.hs = slot;
  if (kVariant == kPessimistic && p.stage < 2) {  // the secondary is read for every key
    p.stage = 2;
    p.skip = true;
  } else {
    p.stage = kDone;
  }
}

// The owner's examination of the line of its current stage (L: the line in the
// warp's slab, sw: its chunk swizzle), and its next stage. A slot's key and
// value sit at key_off / value_off of ckpp_device.cuh: slots below
// first_hi_slot in the first line, the others in the second.
template <int kVariant, bool kCount, int kTM>
__device__ __forceinline__ void examine(Probe& p, const uint8_t* L, uint32_t sw, uint32_t now) {
  if (kVariant == kPessimistic && p.skip) {  // a read made for its cost only
    p.stage = kDone;
    return;
  }
  const bool timers = kTM == kWithTimers || (kTM == kTimersPerKey && p.timers);
  auto chunk = [&](uint32_t c) { return L + 16u * (c ^ sw); };
  auto at = [&](uint32_t byte) { return chunk(byte >> 4) + (byte & 15u); };  // byte offset within the line
  const uint32_t st = p.stage;
  const uint32_t b = st < 2 ? p.b1 : p.b2;
  const uint32_t lo = (1u << first_hi_slot(timers)) - 1u;  // slots of the first line
  const uint32_t base = (st & 1u) ? kLineBytes : 0u;       // this line's first byte in the bucket
  uint32_t cand, alive8;
  if (!(st & 1u)) {  // a bucket's first line: header, then the first slots' entries and the expiries
    const uint4 tg = lds128(chunk(0));
    const uint4 hd = lds128(chunk(1));
    const uint32_t m8 = tag_mask16(tg, p.tag) & hd.z & kBusyMask;
    if (st == 0) {
      const uint64_t bits = (1ull << (p.bidx & 63u)) | (1ull << (p.bidx >> 6));
      p.bloom_ok = (lo64(hd) & bits) == bits;
    }
    alive8 = kBusyMask;
    if (timers) {
      const uint4 ex = lds128(chunk(kExpiryOff / 16u));
      alive8 = alive_mask(lo64(ex), hi64(ex), now);
    }
    cand = m8 & lo;
    p.carry = (m8 & ~lo) | alive8 << 8;  // for the second line, if it is needed
  } else {
    cand = p.carry & 0xFFu;
    alive8 = p.carry >> 8;
  }
  while (cand) {
    const uint32_t s = __ffs(cand) - 1;
    cand &= cand - 1;
    if (kCount) ++p.nrec;
    const uint4 kk = lds128(at(key_off(timers, s) - base));
    if (lo64(kk) == p.k.k0 && hi64(kk) == p.k.k1) {
      if (timers && !((alive8 >> s) & 1u)) {
        resolve<kVariant>(p, false, 0, b, s);  // Sec. 4.2: a dead entry is not returned
      } else {
        resolve<kVariant>(p, true, lds64(at(value_off(timers, s) - base)), b, s);
      }
      return;
    }
  }
  if (!(st & 1u) && (p.carry & 0xFFu)) {  // tag matches in the second line
    p.stage = st + 1;
    return;
  }
  // the bucket does not hold the key
  if (st < 2 && (kVariant != kBloom || p.bloom_ok)) {
    p.stage = 2;
    p.carry = 0;
  } else {
    resolve<kVariant>(p, false, 0, b, 0);
  }
}

// Post p's next line job at position rank of the warp's slab.
template <bool kCount, int G>
__device__ __forceinline__ void post_line(Probe& p, uint32_t rank, WarpStage<G>& S) {
  const uint32_t b = p.stage < 2 ? p.b1 : p.b2;
  S.addr[rank] = reinterpret_cast<unsigned long long>(p.buckets + (uint64_t)b * kBucketBytes +
                                                      (p.stage & 1u) * kLineBytes);
  if (kCount) {
    p.nsec += p.stage == 2;
    p.nline1 += p.stage & 1u;
  }
}

// Copy the nj posted lines into the slab: lane l moves 16-byte chunk l % 8 of
// line 4 i + l / 8 in round i, so each warp instruction requests four whole
// lines. Returns once the warp's copies have landed.
template <int G>
__device__ __forceinline__ void fetch_lines(uint32_t nj, WarpStage<G>& S) {
  const uint32_t lane = threadIdx.x & 31, c = lane & 7u, q = lane >> 3;
  // line j = 4 i + q keeps its chunk c at c ^ (j & 7), and j & 7 = q + 4 (i & 1)
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(&S.line[0][0]) + q * kLineBytes;
  const uint32_t dst_even = base + 16u * (c ^ q), dst_odd = base + 16u * (c ^ (q + 4));
  for (uint32_t i = 0; 4 * i < nj; ++i) {
    const uint32_t j = 4 * i + q;
    if (j < nj) {
      const uint8_t* src = reinterpret_cast<const uint8_t*>(S.addr[j]) + 16u * c;
      const uint32_t dst = ((i & 1u) ? dst_odd : dst_even) + 4 * kLineBytes * i;
      // no L2 hint: evict_last on first lines or evict_first on all lines measured 1-2% slower
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncwarp();
}

// Run the lookups of the warp's lanes until each is resolved. Every lane of
// the warp must call this; lane l owns keys p[0..G) (act[g] false: no key).
template <int kVariant, bool kCount, int G, int kTM>
__device__ __forceinline__ void run_probes(Probe (&p)[G], const bool (&act)[G], uint32_t now, WarpStage<G>& S) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t below = (1u << lane) - 1u;
#pragma unroll
  for (int g = 0; g < G; ++g)
    if (!act[g]) p[g].stage = kDone;
  for (;;) {
    uint32_t rank[G], nj = 0;
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const bool want = p[g].stage < kDone;
      const uint32_t pend = __ballot_sync(kFull, want);
      rank[g] = want ? nj + __popc(pend & below) : 0xFFFFFFFFu;
      nj += __popc(pend);
      if (want) post_line<kCount>(p[g], rank[g], S);
    }
    if (!nj) break;
    __syncwarp();
    fetch_lines(nj, S);
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (rank[g] != 0xFFFFFFFFu) examine<kVariant, kCount, kTM>(p[g], S.line[rank[g]], rank[g] & 7u, now);
    __syncwarp();
  }
}

}  // namespace ckpp
