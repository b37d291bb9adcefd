// Batched insert-or-update (Sec. 2 cuckoo insertion; Sec. 4.1 filter and moved
// counter upkeep; Sec. 4.2 reuse of dead slots).
//
// Kernels, in stream order:
//   dedup   - groups equal keys of the batch in an open-addressing set in the
//             workspace: each key learns the lowest (leader) and highest batch
//             index of its group, which gives the batch the result of inserting
//             the keys one by one in index order. Keys of groups with more than
//             one member are flagged, so a key that occurs once needs no
//             further read of the set.
//   phase1  - per leader, lock-free: update in place if the key is stored
//             (alive; a dead entry is revived), else claim the lowest free
//             or dead slot of the primary, else of the secondary, with a CAS
//             on the bucket's ctrl word, and write the entry into the
//             claimed slot; leaders with two full buckets are queued for the
//             displacement passes.
//   publish - per key: the slot phase 1 claimed becomes busy (one atomic).
//   move1   - per queued leader: the cuckoo paths of length one. Read the
//             entries of b1, then of b2, and the buckets they can move to; the
//             first entry whose other bucket has a free or dead slot moves
//             there under the locks of the path, and the key takes its slot.
//             At load factor 0.9 it places nearly every queued key.
//   phase2  - per key move1 left: breadth-first search for a longer cuckoo
//             path without locks (queue in shared memory), then lock every
//             bucket of the path plus the key's primary, re-validate the path,
//             and move the entries backwards and store the key, all under
//             those locks; retry a bounded number of times. One thread per
//             key, or one warp per key for a short list. Keys still
//             unplaced get a wider search, then the widest, each run by a
//             whole warp per key (a level of the search in two round trips);
//             only then FULL.
//   fixup and finish (one kernel) - reset the filter of buckets whose moved
//             counter reached zero off their lock (the reset of Sec. 4.1,
//             deferred so that it never races a concurrent setter); non-leader
//             occurrences copy their leader's outcome (UPDATED, or FULL/BUSY).
// Before them, one kernel clears the workspace (counters and the dedup set).
// Each kernel after the workspace clear is launched with programmatic stream
// serialization and waits for its predecessor in its first instruction
// (pdl_wait in mutate.cuh), so the GPU schedules it while the predecessor
// drains instead of after it.
#include "mutate.cuh"

namespace ckpp {

namespace {

constexpr int kThreads = 256;
constexpr int kPathAttempts = 16;
// Buckets the one-move pass reads per round trip when looking for room for a root's entries.
constexpr uint32_t kMoveGroup = 2;

__device__ __forceinline__ Key load_key(const uint8_t* keys, uint64_t i) {
  uint64_t a, b;
  asm volatile("ld.global.nc.v2.u64 {%0,%1}, [%2];" : "=l"(a), "=l"(b) : "l"(keys + 16 * i));
  return Key{a, b};
}

// ---------------------------------------------------------------- dedup
// Equal keys bound for different tables are different keys.
__device__ void dedup_one(const uint8_t* __restrict__ keys, const TableSet& ts, const Workspace& ws, uint64_t i) {
  const Key k = load_key(keys, i);
  const uint32_t tid = ts.id(i);
  uint32_t pos = (uint32_t)(hash_key(k, 0x51ED270B27A2B5E3ull ^ tid) >> 16) & ws.m_mask;
  const uint32_t me = (uint32_t)i;
  constexpr unsigned long long kFreePair = kEmpty;  // first kEmpty, last 0
  for (uint32_t probe = 0; probe <= ws.m_mask; ++probe) {
    // one 64-bit CAS claims a free position (first = last = i) or returns the
    // index range of the key group holding it
    unsigned long long* pair = ws.pair_at(pos);
    unsigned long long old = atomicCAS(pair, kFreePair, ((unsigned long long)me << 32) | me);
    if (old == kFreePair) {
      ws.slot_of[i] = pos;
      return;
    }
    // A position only ever holds batch indices of one key group, so the key
    // at index cur is that group's key even while other members widen the range.
    const uint32_t cur = (uint32_t)old;
    const Key o = load_key(keys, cur);
    if (o.k0 == k.k0 && o.k1 == k.k1 && ts.id(cur) == tid) {
      // widen the group's range to include i; a CAS fails only when another
      // member's succeeded, so this ends within the group's size
      for (;;) {
        const uint32_t f = (uint32_t)old, l = (uint32_t)(old >> 32);
        const unsigned long long want = ((unsigned long long)(l > me ? l : me) << 32) | (f < me ? f : me);
        if (want == old) break;
        const unsigned long long seen = atomicCAS(pair, old, want);
        if (seen == old) break;
        old = seen;
      }
      ws.slot_of[i] = pos;
      // both occurrences are flagged: the first to claim the position learns of the
      // group only here (every later occurrence's CAS returns a member of it)
      ws.dup[i] = 1;
      ws.dup[cur] = 1;
      return;
    }
    pos = (pos + 1) & ws.m_mask;
  }
}

__global__ void __launch_bounds__(kThreads) dedup_kernel(const uint8_t* __restrict__ keys, uint64_t n, TableSet ts,
                                                         Workspace ws) {
  pdl_wait();
  pdl_release();
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i < n) dedup_one(keys, ts, ws, i);
}

// The first and last batch index of key i's group: i itself for a key that
// occurs once in the batch (no read of the set), else one 8-byte read.
__device__ __forceinline__ uint2 group_of(const Workspace& ws, uint64_t i) {
  if (!ws.dup[i]) return make_uint2((uint32_t)i, (uint32_t)i);
  return *reinterpret_cast<const uint2*>(ws.first_at(ws.slot_of[i]));
}

__device__ __forceinline__ bool is_leader(const Workspace& ws, uint64_t i, uint32_t& last) {
  const uint2 g = group_of(ws, i);
  if (g.x != (uint32_t)i) return false;
  last = g.y;
  return true;
}

// The value to store for key i: the last occurrence's of its group.
__device__ __forceinline__ uint64_t value_of(const Workspace& ws, const uint64_t* vals, uint64_t i) {
  return vals[group_of(ws, i).y];
}

// Status byte of a key that is not its group's first occurrence, until the
// finishing pass copies its leader's outcome (never returned to the caller).
constexpr uint8_t kStFollower = 0xFF;

// --------------------------------------------------------------- phase 1
// Per leader, without locks. A key that is stored (alive or dead, Sec. 4.2) is
// found in its primary bucket, or in its secondary when the primary's filter
// says it may be there (Sec. 4.1: a key stored in its secondary has both bits
// set in its primary's filter; phase 1 moves no entry and the batch holds each
// key once, so the tests are exact). A live entry is updated in place. Any
// other key claims the lowest claimable slot of its primary, else of its
// secondary (Sec. 2), else waits for the displacement passes.
//
// A claim is a CAS on the bucket's ctrl word that sets the slot's claimed bit
// (and clears its busy and in_secondary bits: a dead entry held there is
// evicted, with moved-counter upkeep on its own primary). A slot is claimable
// if it is neither busy nor claimed, or busy with a dead entry and not
// claimed. The owner then writes the entry; the slot stays invisible to every
// reader, whose searches look at busy slots only, until insert_publish (the
// next kernel) flips its claimed bit to busy. A failed CAS returns the current
// word, and the claimable slots are recomputed from it. Reviving a key's own
// dead entry claims its slot in the same way (busy stays set), so a revival
// and a reuse of that dead slot by another key cannot both succeed. Storing a
// key in its secondary sets its two bits in the primary's filter and counts
// it in the primary's moved counter, with relaxed atomics: no filter is reset
// during phase 1 (resets of counters that reach zero here are deferred to the
// fixup pass). Nothing in phase 1 waits on another thread, and nothing needs
// a fence: the kernel boundary orders every write before the publication.
constexpr int kClaimAttempts = 64;  // CAS retries on one bucket (at most 16 claims can change its word)

__device__ __forceinline__ uint32_t claim_bit(uint32_t s) { return 1u << (kClaimShift + s); }

// Slots of a bucket (ctrl word c, snapshot s) that an insertion may claim.
__device__ __forceinline__ uint32_t claimable(const TableView& t, uint32_t c, const Snap& s, uint32_t now) {
  return free_mask(t, c, s, now) & ~(c >> kClaimShift) & kBusyMask;
}

// Claim the lowest claimable slot of bucket b. c: the word the snapshot s saw.
// Returns the slot (prev receives the word the CAS replaced), -1 if nothing is
// claimable, -2 after kClaimAttempts failed CASes.
__device__ int claim_slot(const TableView& t, uint32_t b, uint32_t c, const Snap& s, uint32_t now, uint32_t& prev) {
  uint32_t* cp = ctrl_ptr(t, b);
  for (int i = 0; i < kClaimAttempts; ++i) {
    const uint32_t f = claimable(t, c, s, now);
    if (!f) return -1;
    const uint32_t sl = __ffs(f) - 1;
    const uint32_t want = (c | claim_bit(sl)) & ~((1u << sl) | (1u << (kInsecShift + sl)));
    const uint32_t got = atomicCAS(cp, c, want);
    if (got == c) {
      prev = c;
      return (int)sl;
    }
    c = got;
  }
  return -2;
}

// Claim the slot of the key's own dead entry (slot sl of bucket b, busy in c).
// Returns 1 on success, 0 if another key took the slot first (the entry is
// gone), -2 after kClaimAttempts failed CASes.
__device__ int claim_revival(const TableView& t, uint32_t b, uint32_t sl, uint32_t c) {
  uint32_t* cp = ctrl_ptr(t, b);
  for (int i = 0; i < kClaimAttempts; ++i) {
    if (!((c >> sl) & 1u) || ((c >> (kClaimShift + sl)) & 1u)) return 0;
    const uint32_t got = atomicCAS(cp, c, c | claim_bit(sl));
    if (got == c) return 1;
    c = got;
  }
  return -2;
}

// A dead entry evicted by a claim (prev: the word before it): if it sat in its
// secondary bucket, its primary's moved counter drops (Sec. 4.1); a counter
// that reaches zero is queued for the filter reset of the fixup pass.
__device__ __forceinline__ void evict_claimed(const TableView& t, uint32_t tid, uint32_t b, uint32_t sl,
                                             uint32_t prev, const Workspace& ws) {
  if (((prev >> sl) & 1u) && ((prev >> (kInsecShift + sl)) & 1u)) {
    Key k;
    ld128_cg(key_ptr(t, b, sl), k.k0, k.k1);
    const Addr e = address_of(k, t.nb, t.seed);
    if (atomicSub(moved_ptr(t, e.b1), 1u) == 1u) push_fixup(ws, tid, e.b1);
  }
}

struct P1Result {
  uint8_t status;           // 0: queued for the displacement passes
  unsigned long long rec;   // the claim to publish, or 0
};

// The key's stored entry in bucket b (snapshot s, word c), if any: a live one
// is updated in place (UPDATED), a dead one revived through a claim
// (INSERTED, Sec. 4.2). Returns false if the key is not there (or its dead
// entry was just taken by another key).
__device__ bool update_stored(const TableView& t, uint32_t b, uint32_t c, const Snap& s, const Key& k,
                              const Addr& a, uint64_t v, uint32_t now, uint32_t expiry, P1Result& r) {
  const int slot = find_key(t, b, c, s, k, a.tag);
  if (slot < 0) return false;
  if (!t.timers || alive16(snap_expiry(s, slot), now)) {
    st64_cg(value_ptr(t, b, slot), v);
    if (t.timers) set_expiry(t, b, slot, expiry);
    r.status = kStUpdated;
    return true;
  }
  const int got = claim_revival(t, b, (uint32_t)slot, c);
  if (got == 0) return false;
  if (got < 0) {
    r.status = kStBusy;
    return true;
  }
  st64_cg(value_ptr(t, b, slot), v);
  set_expiry(t, b, slot, expiry);
  r.status = kStInserted;
  r.rec = ((unsigned long long)b << 32) | claim_bit(slot);
  return true;
}

// Claim a slot of bucket b for the new key and write its entry there.
// Returns false if b has nothing claimable.
__device__ bool place_new(const TableView& t, uint32_t tid, uint32_t b, uint32_t c, const Snap& s, const Key& k,
                          const Addr& a, uint64_t v, uint32_t now, uint32_t expiry, const Workspace& ws,
                          P1Result& r) {
  uint32_t prev = 0;
  const int sl = claim_slot(t, b, c, s, now, prev);
  if (sl == -1) return false;
  if (sl < 0) {
    r.status = kStBusy;
    return true;
  }
  evict_claimed(t, tid, b, (uint32_t)sl, prev, ws);
  st128_cg(key_ptr(t, b, sl), k.k0, k.k1);
  st64_cg(value_ptr(t, b, sl), v);
  st16_cg(tag_ptr(t, b, sl), a.tag);
  if (t.timers) st16_cg(expiry_ptr(t, b, sl), expiry);
  uint32_t flip = claim_bit(sl) | (1u << sl);
  if (b == a.b2) {  // Sec. 4.1: displaced to the secondary
    flip |= 1u << (kInsecShift + sl);
    atomicOr(reinterpret_cast<unsigned long long*>(bloom_ptr(t, a.b1)), (unsigned long long)a.bits);
    atomicAdd(moved_ptr(t, a.b1), 1u);
  }
  r.status = kStInserted;
  r.rec = ((unsigned long long)b << 32) | flip;
  return true;
}

__device__ void phase1_one(const TableSet& ts, const uint8_t* __restrict__ keys, const uint64_t* __restrict__ vals,
                           uint32_t now, uint32_t expiry, uint8_t* __restrict__ status, const Workspace& ws,
                           uint64_t i) {
  P1Result r{0, 0ull};
  // The leader test's set words and the primary's snapshot are independent
  // round trips; both are requested before either is used.
  const uint2 g = group_of(ws, i);
  const uint32_t first = g.x, last = g.y;
  if (!ts.valid(i)) {
    ws.claim[i] = 0ull;
    status[i] = first == (uint32_t)i ? kStNoTable : kStFollower;
    return;
  }
  const TableView t = ts.of(i);
  const uint32_t tid = ts.id(i);
  const Key k = load_key(keys, i);
  const Addr a = address_of(k, t.nb, t.seed);
  Snap s1, s2;
  snap_bucket(t, a.b1, s1);
  if (first != (uint32_t)i) {
    ws.claim[i] = 0ull;
    status[i] = kStFollower;
    return;
  }
  const uint64_t v = vals[last];
  const uint32_t c1 = (uint32_t)s1.w[3];
  bool done = update_stored(t, a.b1, c1, s1, k, a, v, now, expiry, r);
  bool have2 = false;
  uint32_t c2 = 0;
  if (!done && (s1.w[2] & a.bits) == a.bits) {  // the filter allows the secondary
    snap_bucket(t, a.b2, s2);
    have2 = true;
    c2 = (uint32_t)s2.w[3];
    done = update_stored(t, a.b2, c2, s2, k, a, v, now, expiry, r);
  }
  if (!done) done = place_new(t, tid, a.b1, c1, s1, k, a, v, now, expiry, ws, r);
  if (!done) {
    if (!have2) {
      snap_bucket(t, a.b2, s2);
      c2 = (uint32_t)s2.w[3];
    }
    done = place_new(t, tid, a.b2, c2, s2, k, a, v, now, expiry, ws, r);
  }
  ws.claim[i] = r.rec;
  if (!done) {
    ws.pending[atomicAdd(ws.counters + 0, 1u)] = (uint32_t)i;
    return;
  }
  if (r.status == kStBusy) latch_error(t, kErrLockTimeout);
  status[i] = r.status;
}

__global__ void __launch_bounds__(kThreads, 1) insert_phase1(TableSet ts, const uint8_t* __restrict__ keys,
                                                          const uint64_t* __restrict__ vals, uint64_t n,
                                                          uint32_t now, uint32_t expiry, uint8_t* __restrict__ status,
                                                          Workspace ws) {
  pdl_wait();
  pdl_release();
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i < n) phase1_one(ts, keys, vals, now, expiry, status, ws, i);
}

// Publication of phase 1's claims: each claimed slot's claimed bit is cleared
// and its busy (and in_secondary) bits set, in one atomic XOR per key. From
// here on the new entries are visible to every search.
__device__ __forceinline__ void publish_one(const TableSet& ts, const Workspace& ws, uint64_t i) {
  const unsigned long long r = ws.claim[i];
  if (!r) return;
  const TableView t = ts.of(i);
  atomicXor(ctrl_ptr(t, (uint32_t)(r >> 32)), (uint32_t)r);
}

__global__ void __launch_bounds__(kThreads) insert_publish(TableSet ts, uint64_t n, Workspace ws) {
  pdl_wait();
  pdl_release();
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i < n) publish_one(ts, ws, i);
}

// --------------------------------------------------------------- phase 2
// Search budgets of the displacement passes after move1 (queue in shared
// memory, at most 48 KB per block): the grid pass searches 96 buckets up to 4
// moves deep, one thread per key (many keys, so the searches in flight matter
// most; a list of at most kGridWarpKeys keys runs one warp per key); the
// second pass 192 buckets, 5 moves, and the last pass 2048 buckets, 6 moves,
// one warp per key (few keys, so the time of one search matters most; the
// sequential CPU reference searches 1024 buckets, 5 moves). Each
// later pass takes on at most kSecondPassKeys / kLastPassKeys keys, which
// bounds the time a batch spends on a table that is full: the rest are FULL
// without a search. Near LF 0.98 the second pass still places about two
// thirds of the keys it searches, so its share is wide.
//
// Within one insert call no bucket gains a free or dead slot: phase 1 fills
// them, a path ends by filling one, every move along it vacates a slot that
// the next move (or the key) refills, and `now` is fixed. A key queued by
// phase 1 found both its buckets without a free or dead slot, so the passes
// search from them without re-checking the roots.
constexpr int kP2Threads = 64;
constexpr uint32_t kSecondPassKeys = 65536;  // keys the second pass takes on
constexpr uint32_t kLastPassKeys = 1024;     // keys the last pass takes on
// A grid search list this short runs one warp per key: the slowest search sets
// the pass's time, and a warp takes a level of a search in two round trips.
constexpr uint32_t kGridWarpKeys = 1024;
constexpr int kMaxDepth = 6;
constexpr int kPathBuckets = kMaxDepth + 1;
constexpr int kMaxLocks = kPathBuckets + 1;   // the path plus the key's primary

struct Node {
  uint32_t bucket;
  int16_t parent;
  uint8_t slot;   // slot of the parent bucket whose entry moves into this bucket
  uint8_t depth;
};

// One thread's search queue inside a block's shared array stored node-major
// (node j of every thread side by side), so that the threads of a warp touch
// consecutive words and never the same bank.
struct Queue {
  Node* base;
  int stride;
  __device__ __forceinline__ Node& operator[](int i) const { return base[i * stride]; }
};

// Breadth-first search over buckets from b1 and b2 by one thread (lock-free
// reads; the path is re-validated under its locks). Expanding a bucket issues
// the reads of its control word and the keys of its 8 slots together (each
// entry's other bucket takes one hash, chosen by its in_secondary bit), then
// the control-word (and expiry) reads of the 8 buckets those entries can move
// to, so one level of the search costs two memory round trips; a child with a
// free or dead slot ends the search (the first such child in queue order, i.e.
// a shortest path). A child is not queued if it is one of the roots, a bucket
// on its parent's path or an earlier sibling, so no path holds a bucket twice;
// a bucket reached again by another branch takes a second queue node (a scan
// of the whole queue for it cost more than the node: most repeats are an
// entry's way back to the bucket it came from, which the path test catches).
// Returns the node index of the bucket with the hole (in hole), or -1.
template <int kBfsNodes, int kBfsDepth>
__device__ int bfs(const TableView& t, const Addr& a, uint32_t now, const Queue& q, uint32_t& hole) {
  static_assert(kBfsNodes < 32768, "parent index exceeds its field");
  int nq = 0;
  q[nq++] = Node{a.b1, -1, 0, 0};
  q[nq++] = Node{a.b2, -1, 0, 0};
  // A hole is only ever found on a newly queued bucket, so the search ends
  // when the queue is full.
  for (int qi = 0; qi < nq && nq < kBfsNodes; ++qi) {
    const Node cur = q[qi];
    if (cur.depth >= kBfsDepth) continue;
    uint64_t k0[kSlots], k1[kSlots];
    const uint32_t cc = load_bucket_keys(t, cur.bucket, k0, k1);
    uint32_t y[kSlots], cy[kSlots];
    uint64_t e0[kSlots], e1[kSlots];
#pragma unroll
    for (uint32_t sl = 0; sl < kSlots; ++sl)
      y[sl] = other_bucket(Key{k0[sl], k1[sl]}, cur.bucket, (cc >> (kInsecShift + sl)) & 1u, t.nb, t.seed);
#pragma unroll
    for (uint32_t sl = 0; sl < kSlots; ++sl) {
      cy[sl] = ld32_cg(ctrl_ptr(t, y[sl]));
      if (t.timers) {
        ld128_cg(expiry_ptr(t, y[sl], 0), e0[sl], e1[sl]);
      } else {
        e0[sl] = e1[sl] = 0;
      }
    }
    // children to skip: a root, a bucket on cur's path (cur and its ancestors), an earlier sibling
    uint32_t path_b[kBfsDepth + 1];
    int node = qi;
#pragma unroll
    for (int d = 0; d <= kBfsDepth; ++d) {
      path_b[d] = node >= 0 ? q[node].bucket : a.b1;  // past the root: a root again, already tested
      node = node >= 0 ? q[node].parent : -1;
    }
    uint32_t skip = 0;
#pragma unroll
    for (uint32_t sl = 0; sl < kSlots; ++sl) {
      bool hit = y[sl] == a.b1 || y[sl] == a.b2;
#pragma unroll
      for (int d = 0; d <= kBfsDepth; ++d) hit |= path_b[d] == y[sl];
#pragma unroll
      for (uint32_t o = 0; o < sl; ++o) hit |= y[o] == y[sl];
      skip |= (uint32_t)hit << sl;
    }
    for (uint32_t sl = 0; sl < kSlots && nq < kBfsNodes; ++sl) {
      if ((skip >> sl) & 1u) continue;
      q[nq] = Node{y[sl], (int16_t)qi, (uint8_t)sl, (uint8_t)(cur.depth + 1)};
      Snap s;
      s.e0 = e0[sl];
      s.e1 = e1[sl];
      const uint32_t f = free_mask(t, cy[sl], s, now);
      ++nq;
      if (f) {
        hole = __ffs(f) - 1;
        return nq - 1;
      }
    }
  }
  return -1;
}

// The same search run by a whole warp for one key. A round expands up to 32
// queued buckets at once, one per lane, with the thread form's two round trips
// (a lane's bucket keys and control word, then the control words of the 8
// buckets its entries can move to), so a level of the search costs two round
// trips however wide it is. The children of a round enter the queue in queue
// order (lane, then slot; the queue stays sorted by depth), each bucket once:
// the visited set is a shared open-addressing table updated with atomicCAS,
// sized for the queue plus one round of children. The hole is the first child
// in queue order with a free or dead slot, a shortest path as in the thread
// form. q: the warp's queue (kBfsNodes nodes); seen: its set. Every lane
// returns the same node index (or -1) and hole.
constexpr uint32_t kWarpAll = 0xFFFFFFFFu;

template <int kBfsNodes>
struct WarpSeen {
  // smallest power of two at least 1.5 x (kBfsNodes + the 256 children of a round)
  static constexpr uint32_t kNeed = (kBfsNodes + 256) * 3 / 2;
  static constexpr uint32_t kSize = kNeed <= 1024 ? 1024 : (kNeed <= 2048 ? 2048 : (kNeed <= 4096 ? 4096 : 8192));
  static_assert(kNeed <= 8192, "visited set too large");
};

template <uint32_t kSize>
__device__ __forceinline__ bool seen_insert_shared(uint32_t* seen, uint32_t b) {
  uint32_t h = (b * 0x9E3779B1u) & (kSize - 1);
  for (uint32_t probe = 0; probe < kSize; ++probe) {
    const uint32_t old = atomicCAS(&seen[h], 0xFFFFFFFFu, b);
    if (old == 0xFFFFFFFFu) return true;
    if (old == b) return false;
    h = (h + 1) & (kSize - 1);
  }
  return false;  // not reached: the set is sized for every bucket a search can meet
}

template <int kBfsNodes, int kBfsDepth>
__device__ int bfs_warp(const TableView& t, const Addr& a, uint32_t now, Node* q, uint32_t* seen, uint32_t& hole) {
  constexpr uint32_t kSeen = WarpSeen<kBfsNodes>::kSize;
  const uint32_t lane = threadIdx.x & 31u;
  for (uint32_t j = lane; j < kSeen; j += 32) seen[j] = 0xFFFFFFFFu;
  __syncwarp();
  if (lane == 0) {
    q[0] = Node{a.b1, -1, 0, 0};
    q[1] = Node{a.b2, -1, 0, 0};
    seen_insert_shared<kSeen>(seen, a.b1);
    seen_insert_shared<kSeen>(seen, a.b2);
  }
  __syncwarp();
  int nq = 2;
  for (int head = 0; head < nq && nq < kBfsNodes;) {
    const int chunk_end = min(nq, head + 32);
    const int qi = head + (int)lane;
    Node cur{0, -1, 0, (uint8_t)kBfsDepth};
    if (qi < chunk_end) cur = q[qi];
    uint32_t y[kSlots];
    uint32_t fresh = 0;   // children this lane queues
    uint64_t holes = 0;   // their free or dead slots, 8 bits per child
    if (cur.depth < kBfsDepth) {
      uint64_t k0[kSlots], k1[kSlots];
      const uint32_t cc = load_bucket_keys(t, cur.bucket, k0, k1);
      uint32_t cy[kSlots];
      uint64_t e0[kSlots], e1[kSlots];
#pragma unroll
      for (uint32_t sl = 0; sl < kSlots; ++sl)
        y[sl] = other_bucket(Key{k0[sl], k1[sl]}, cur.bucket, (cc >> (kInsecShift + sl)) & 1u, t.nb, t.seed);
#pragma unroll
      for (uint32_t sl = 0; sl < kSlots; ++sl) {
        cy[sl] = ld32_cg(ctrl_ptr(t, y[sl]));
        if (t.timers) {
          ld128_cg(expiry_ptr(t, y[sl], 0), e0[sl], e1[sl]);
        } else {
          e0[sl] = e1[sl] = 0;
        }
      }
#pragma unroll
      for (uint32_t sl = 0; sl < kSlots; ++sl) {
        if (!seen_insert_shared<kSeen>(seen, y[sl])) continue;
        fresh |= 1u << sl;
        Snap s;
        s.e0 = e0[sl];
        s.e1 = e1[sl];
        holes |= (uint64_t)free_mask(t, cy[sl], s, now) << (8 * sl);
      }
    }
    // queue positions: the children of lower lanes first
    const uint32_t cnt = __popc(fresh);
    uint32_t incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(kWarpAll, incl, d);
      if ((int)lane >= d) incl += o;
    }
    const uint32_t total = __shfl_sync(kWarpAll, incl, 31);
    int pos = nq + (int)(incl - cnt);
    int best = 0x7FFFFFFF;  // this lane's first queued child with room
    uint32_t best_hole = 0;
#pragma unroll
    for (uint32_t sl = 0; sl < kSlots; ++sl) {
      if (!((fresh >> sl) & 1u)) continue;
      if (pos < kBfsNodes) {
        q[pos] = Node{y[sl], (int16_t)qi, (uint8_t)sl, (uint8_t)(cur.depth + 1)};
        const uint32_t f = (uint32_t)(holes >> (8 * sl)) & 0xFFu;
        if (f && best == 0x7FFFFFFF) {
          best = pos;
          best_hole = __ffs(f) - 1;
        }
      }
      ++pos;
    }
    __syncwarp();  // the new nodes before any lane reads them
    const int wbest = __reduce_min_sync(kWarpAll, best);
    if (wbest != 0x7FFFFFFF) {
      const uint32_t src = __ffs(__ballot_sync(kWarpAll, best == wbest)) - 1;
      hole = __shfl_sync(kWarpAll, best_hole, src);
      return wbest;
    }
    nq = min(nq + (int)total, kBfsNodes);
    head = chunk_end;
  }
  return -1;
}

// Move the entry in slot sx of locked bucket x to the free slot sy of locked
// bucket y, its other bucket. Sec. 4.1: a move from the primary to the
// secondary sets the entry's bits in the primary's filter and increments its
// counter; the reverse move decrements the counter and resets the filter at
// zero (safe: filter bits of y are only ever set under y's lock, held here).
__device__ void move_locked(const TableView& t, uint32_t x, uint32_t sx, uint32_t& cx, uint32_t y, uint32_t sy,
                            uint32_t& cy) {
  uint64_t k0, k1;
  ld128_cg(key_ptr(t, x, sx), k0, k1);
  const uint64_t v = ld64_cg(value_ptr(t, x, sx));
  const Addr e = address_of(Key{k0, k1}, t.nb, t.seed);
  st128_cg(key_ptr(t, y, sy), k0, k1);
  st64_cg(value_ptr(t, y, sy), v);
  st16_cg(tag_ptr(t, y, sy), e.tag);
  if (t.timers) st16_cg(expiry_ptr(t, y, sy), ld16_cg(expiry_ptr(t, x, sx)));
  cy |= 1u << sy;
  if (e.b1 == x) {
    cy |= 1u << (kInsecShift + sy);
    atomicOr(reinterpret_cast<unsigned long long*>(bloom_ptr(t, x)), (unsigned long long)e.bits);
    atomicAdd(moved_ptr(t, x), 1u);
  } else {
    cy &= ~(1u << (kInsecShift + sy));
    if (atomicSub(moved_ptr(t, y), 1u) == 1u) atomicExch(reinterpret_cast<unsigned long long*>(bloom_ptr(t, y)), 0ull);
  }
  cx &= ~((1u << sx) | (1u << (kInsecShift + sx)));
}

// Execute a cuckoo path atomically: lock every bucket on it plus the key's
// primary (in index order), check that each entry still sits where the search
// saw it and still has the next bucket as its other bucket and that the end
// slot is still free or dead, then move the entries backwards (each into the
// hole ahead of it) and store the new key in the hole left in the root bucket.
// path[0] is the root (b1 or b2), path[len] the bucket with the hole; slot[j]
// is the slot of path[j] whose entry moves to path[j + 1].
// 1 placed, 0 stale path, -1 lock timeout.
__device__ int execute_path(const TableView& t, uint32_t tid, const uint32_t (&path)[kPathBuckets],
                            const uint32_t (&slot)[kPathBuckets], int len, uint32_t hole, const Key& k, uint64_t v,
                            const Addr& a, uint32_t now, uint32_t expiry, const Workspace& ws) {
  uint32_t lk[kMaxLocks], cw[kMaxLocks];
  int nl = 0;
  bool has_b1 = false;
  for (int j = 0; j <= len; ++j) {
    lk[nl++] = path[j];
    has_b1 |= (path[j] == a.b1);
  }
  if (!has_b1) lk[nl++] = a.b1;
  for (int i = 1; i < nl; ++i)  // insertion sort: a global lock order
    for (int j = i; j > 0 && lk[j - 1] > lk[j]; --j) {
      const uint32_t tmp = lk[j];
      lk[j] = lk[j - 1];
      lk[j - 1] = tmp;
    }
  for (int i = 0; i < nl; ++i) {
    if (!lock_bucket(t, lk[i], cw[i])) {
      for (int j = i - 1; j >= 0; --j) unlock_bucket(t, lk[j], cw[j]);
      return -1;
    }
  }
  auto idx = [&](uint32_t b) {
    int r = 0;
    for (int i = 0; i < nl; ++i) r = (lk[i] == b) ? i : r;
    return r;
  };
  bool ok = true;
  for (int j = 0; j < len && ok; ++j) {
    if (!((cw[idx(path[j])] >> slot[j]) & 1u)) {
      ok = false;
      break;
    }
    Key ek;
    ld128_cg(key_ptr(t, path[j], slot[j]), ek.k0, ek.k1);
    const Addr e = address_of(ek, t.nb, t.seed);
    const uint32_t other = (e.b1 == path[j]) ? e.b2 : (e.b2 == path[j] ? e.b1 : 0xFFFFFFFFu);
    ok = (other == path[j + 1]);
  }
  const int ie = idx(path[len]);
  const bool end_busy = (cw[ie] >> hole) & 1u;
  if (ok && end_busy) ok = t.timers && !alive16(ld16_cg(expiry_ptr(t, path[len], hole)), now);
  int rc = 0;
  if (ok) {
    if (end_busy) evict_entry(t, tid, path[len], hole, cw[ie], ws);
    uint32_t dst_s = hole;
    for (int j = len - 1; j >= 0; --j) {
      move_locked(t, path[j], slot[j], cw[idx(path[j])], path[j + 1], dst_s, cw[idx(path[j + 1])]);
      dst_s = slot[j];
    }
    place_entry(t, path[0], dst_s, k, v, a, expiry, cw[idx(path[0])]);
    rc = 1;
  }
  for (int i = nl - 1; i >= 0; --i) unlock_bucket(t, lk[i], cw[i]);
  return rc;
}

// A cuckoo path of length one, found by the one-move pass: the entry in slot
// sx of root x (a root of key k: a.b1 or a.b2) moves to free (or dead) slot
// hole of its other bucket y, and k takes slot sx. Under the locks of x, y and
// (when x is k's secondary) k's primary, the path is valid if slot sx is busy
// and its entry's other bucket, from the key and in_secondary bit read under
// the locks, is still y, and y still has room: the hole if it is still free or
// dead, else any slot of y that is free now. The entry's value
// and expiry are read in the same round trip as its key; its tag and filter
// bits come from its two hashes. The moves are those of execute_path. 1
// placed, 0 stale path, -1 lock timeout.
__device__ int execute_move1(const TableView& t, uint32_t tid, uint32_t x, uint32_t sx, uint32_t y, uint32_t hole,
                             const Key& k, uint64_t v, const Addr& a, uint32_t now, uint32_t expiry,
                             const Workspace& ws) {
  uint32_t lk[3], cw[3];
  int nl = 0;
  // x and y are distinct and differ from a.b1 unless x == a.b1 (the search skips y in {b1, b2})
  const uint32_t u0 = x < y ? x : y, u1 = x < y ? y : x;
  if (x == a.b1) {
    lk[0] = u0;
    lk[1] = u1;
    nl = 2;
  } else {
    const uint32_t p = a.b1;
    lk[0] = p < u0 ? p : u0;
    lk[1] = p < u0 ? u0 : (p < u1 ? p : u1);
    lk[2] = p < u1 ? u1 : p;
    nl = 3;
  }
  if (!lock_buckets<3>(t, lk, nl, cw)) return -1;
  int ix = 0, iy = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (i < nl && lk[i] == x) ix = i;
    if (i < nl && lk[i] == y) iy = i;
  }
  Key ek;
  ld128_cg(key_ptr(t, x, sx), ek.k0, ek.k1);
  const uint64_t ev = ld64_cg(value_ptr(t, x, sx));
  const uint32_t eexp = t.timers ? ld16_cg(expiry_ptr(t, x, sx)) : 0u;
  const uint32_t hexp = t.timers ? ld16_cg(expiry_ptr(t, y, hole)) : 0u;
  const bool insec = (cw[ix] >> (kInsecShift + sx)) & 1u;
  // H1 gives the entry's tag and the primary of an entry in its secondary, H2 the secondary
  // (and filter bits) of an entry in its primary; hashing beats a fourth memory request
  const uint64_t h1 = hash_key(ek, t.seed), h2 = hash_key(ek, t.seed ^ kSeed2Xor);
  const uint32_t b2 = reduce(h2, t.nb);
  const uint32_t other = insec ? reduce(h1, t.nb) : (b2 != x ? b2 : (x + 1 == (uint32_t)t.nb ? 0u : x + 1));
  const uint32_t etag = (uint32_t)(h1 & 0xFFFF);
  const uint64_t bits = (1ull << (h2 & 63)) | (1ull << ((h2 >> 6) & 63));
  bool ok = ((cw[ix] >> sx) & 1u) && other == y;
  bool end_busy = (cw[iy] >> hole) & 1u;
  if (end_busy && !(t.timers && !alive16(hexp, now))) {
    // another key took the hole since the search: any slot of y that is free now will do
    const uint32_t fr = ~cw[iy] & kBusyMask;
    if (fr) {
      hole = __ffs(fr) - 1;
      end_busy = false;
    }
  }
  if (ok && end_busy) ok = t.timers && !alive16(hexp, now);
  if (ok) {
    if (end_busy) evict_entry(t, tid, y, hole, cw[iy], ws);
    st128_cg(key_ptr(t, y, hole), ek.k0, ek.k1);
    st64_cg(value_ptr(t, y, hole), ev);
    st16_cg(tag_ptr(t, y, hole), etag);
    if (t.timers) st16_cg(expiry_ptr(t, y, hole), eexp);
    cw[iy] |= 1u << hole;
    if (!insec) {  // Sec. 4.1: primary x -> secondary y: x's filter gets the entry's bits, its counter + 1
      cw[iy] |= 1u << (kInsecShift + hole);
      atomicOr(reinterpret_cast<unsigned long long*>(bloom_ptr(t, x)), (unsigned long long)bits);
      atomicAdd(moved_ptr(t, x), 1u);
    } else {  // secondary x -> primary y: y's counter - 1, its filter reset at zero (y is locked)
      cw[iy] &= ~(1u << (kInsecShift + hole));
      if (atomicSub(moved_ptr(t, y), 1u) == 1u) atomicExch(reinterpret_cast<unsigned long long*>(bloom_ptr(t, y)), 0ull);
    }
    cw[ix] &= ~((1u << sx) | (1u << (kInsecShift + sx)));
    place_entry(t, x, sx, k, v, a, expiry, cw[ix]);
  }
  unlock_buckets<3>(t, lk, nl, cw);
  return ok ? 1 : 0;
}

// One-move pass over `list` (count in *count_ptr): for each key, the entries
// of b1 and then of b2 are read with the buckets they can move to (two memory
// round trips per root: the root's keys and control word, then the control
// words of the buckets its entries can move to; each entry's other bucket
// takes one hash, chosen by its in_secondary bit); the first entry whose other
// bucket has a free or dead slot gives a cuckoo path of length one, executed
// under locks (execute_move1). Keys without one, or whose path went stale, are
// appended to `next`. The key's value is requested before the search.
// worker / workers: this thread's index among the threads sharing the pass.
__device__ void move1_range(const TableSet& ts, const uint8_t* __restrict__ keys, const uint64_t* __restrict__ vals,
                            uint32_t now, uint32_t expiry, uint8_t* __restrict__ status, const Workspace& ws,
                            const uint32_t* list, const uint32_t* count_ptr, uint32_t* next, uint32_t* next_count,
                            uint32_t worker, uint32_t workers) {
  const uint32_t count = ld32_cg(count_ptr);
  for (uint32_t j = worker; j < count; j += workers) {
    const uint32_t i = list[j];
    const TableView t = ts.of(i);
    const uint64_t v = value_of(ws, vals, i);
    const Key k = load_key(keys, i);
    const Addr a = address_of(k, t.nb, t.seed);
    uint32_t x = 0, sx = 0, y = 0, hole = 0;
    bool found = false;
    for (int r = 0; r < 2 && !found; ++r) {
      const uint32_t root = r ? a.b2 : a.b1;
      uint64_t k0[kSlots], k1[kSlots];
      const uint32_t cr = load_bucket_keys(t, root, k0, k1);
      uint32_t yy[kSlots];
#pragma unroll
      for (uint32_t sl = 0; sl < kSlots; ++sl)
        yy[sl] = other_bucket(Key{k0[sl], k1[sl]}, root, (cr >> (kInsecShift + sl)) & 1u, t.nb, t.seed);
      // the buckets the entries can move to, kMoveGroup at a time: most keys find room among the
      // first ones, and each bucket read is a memory request of its own
      for (uint32_t g = 0; g < kSlots && !found; g += kMoveGroup) {
        uint32_t cy[kMoveGroup];
        uint64_t e0[kMoveGroup], e1[kMoveGroup];
#pragma unroll
        for (uint32_t q = 0; q < kMoveGroup; ++q) {
          cy[q] = ld32_cg(ctrl_ptr(t, yy[g + q]));
          if (t.timers) {
            ld128_cg(expiry_ptr(t, yy[g + q], 0), e0[q], e1[q]);
          } else {
            e0[q] = e1[q] = 0;
          }
        }
#pragma unroll
        for (uint32_t q = 0; q < kMoveGroup; ++q) {
          const uint32_t sl = g + q;
          if (found || yy[sl] == a.b1 || yy[sl] == a.b2) continue;  // the roots have no room
          Snap s;
          s.e0 = e0[q];
          s.e1 = e1[q];
          const uint32_t f = free_mask(t, cy[q], s, now);
          if (f) {
            x = root;
            sx = sl;
            y = yy[sl];
            hole = __ffs(f) - 1;
            found = true;
          }
        }
      }
    }
    int rc = 0;
    if (found) rc = execute_move1(t, ts.id(i), x, sx, y, hole, k, v, a, now, expiry, ws);
    if (rc == 0) {
      next[atomicAdd(next_count, 1u)] = i;
    } else {
      if (rc < 0) latch_error(t, kErrLockTimeout);
      status[i] = rc > 0 ? kStInserted : kStBusy;
    }
  }
}

__global__ void __launch_bounds__(kThreads) insert_move1(TableSet ts, const uint8_t* __restrict__ keys,
                                                         const uint64_t* __restrict__ vals, uint32_t now,
                                                         uint32_t expiry, uint8_t* __restrict__ status, Workspace ws,
                                                         const uint32_t* list, const uint32_t* count_ptr,
                                                         uint32_t* next, uint32_t* next_count) {
  pdl_wait();
  pdl_release();
  move1_range(ts, keys, vals, now, expiry, status, ws, list, count_ptr, next, next_count,
              blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// Displacement pass over `list` (count in *count). Keys that find no path
// are appended to `retry` (when given) for a second, low-contention pass;
// otherwise they are FULL. q: this thread's search queue.
template <int kBfsNodes, int kBfsDepth>
__device__ void phase2_range(const TableSet& ts, const uint8_t* __restrict__ keys, const uint64_t* __restrict__ vals,
                             uint32_t now, uint32_t expiry, uint8_t* __restrict__ status, const Workspace& ws,
                             const uint32_t* list, uint32_t listed, uint32_t* retry, uint32_t* retry_count,
                             uint32_t max_keys, const Queue& q, uint32_t worker, uint32_t workers) {
  static_assert(kBfsDepth <= kMaxDepth, "path longer than the lock set");
  const uint32_t count = min(listed, max_keys);
  // A later pass searches wider but alone; when many keys reach it the table
  // is full rather than contended, and those beyond max_keys are FULL at once.
  for (uint32_t j = count + worker; j < listed; j += workers) status[list[j]] = kStFull;
  for (uint32_t j = worker; j < count; j += workers) {
    const uint32_t i = list[j];
    const TableView t = ts.of(i);
    const uint32_t tid = ts.id(i);
    const uint64_t v = value_of(ws, vals, i);
    const Key k = load_key(keys, i);
    const Addr a = address_of(k, t.nb, t.seed);
    uint8_t st = kStFull;
    for (int attempt = 0; attempt < kPathAttempts; ++attempt) {
      uint32_t hole = 0;
      const int end = bfs<kBfsNodes, kBfsDepth>(t, a, now, q, hole);
      if (end < 0) break;  // no cuckoo path within the search bound: FULL
      uint32_t path[kPathBuckets], slot[kPathBuckets];
      const int len = q[end].depth;
      for (int node = end; node >= 0; node = q[node].parent) {
        path[q[node].depth] = q[node].bucket;
        if (q[node].depth > 0) slot[q[node].depth - 1] = q[node].slot;
      }
      const int r = execute_path(t, tid, path, slot, len, hole, k, v, a, now, expiry, ws);
      if (r != 0) {
        st = r > 0 ? kStInserted : kStBusy;
        break;
      }
    }
    if (st == kStFull && retry) {
      retry[atomicAdd(retry_count, 1u)] = i;
      continue;
    }
    if (st == kStBusy) latch_error(t, kErrLockTimeout);
    status[i] = st;
  }
}

// phase2_range with one warp per key (bfs_warp): warp / warps are this warp's
// index among the warps sharing the pass; q and seen are the warp's own.
// listed: the list's length (read by the caller after the list was final).
template <int kBfsNodes, int kBfsDepth>
__device__ void phase2_range_warp(const TableSet& ts, const uint8_t* __restrict__ keys,
                                  const uint64_t* __restrict__ vals, uint32_t now, uint32_t expiry,
                                  uint8_t* __restrict__ status, const Workspace& ws, const uint32_t* list,
                                  uint32_t listed, uint32_t* retry, uint32_t* retry_count,
                                  uint32_t max_keys, Node* q, uint32_t* seen, uint32_t warp, uint32_t warps) {
  static_assert(kBfsDepth <= kMaxDepth, "path longer than the lock set");
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t count = min(listed, max_keys);
  for (uint32_t j = count + warp * 32 + lane; j < listed; j += warps * 32) status[list[j]] = kStFull;
  for (uint32_t j = warp; j < count; j += warps) {
    const uint32_t i = list[j];
    const TableView t = ts.of(i);
    const uint32_t tid = ts.id(i);
    const uint64_t v = value_of(ws, vals, i);
    const Key k = load_key(keys, i);
    const Addr a = address_of(k, t.nb, t.seed);
    uint8_t st = kStFull;
    for (int attempt = 0; attempt < kPathAttempts; ++attempt) {
      uint32_t hole = 0;
      const int end = bfs_warp<kBfsNodes, kBfsDepth>(t, a, now, q, seen, hole);
      if (end < 0) break;  // no cuckoo path within the search bound: FULL
      int r = 0;
      if (lane == 0) {
        uint32_t path[kPathBuckets], slot[kPathBuckets];
        const int len = q[end].depth;
        for (int node = end; node >= 0; node = q[node].parent) {
          path[q[node].depth] = q[node].bucket;
          if (q[node].depth > 0) slot[q[node].depth - 1] = q[node].slot;
        }
        r = execute_path(t, tid, path, slot, len, hole, k, v, a, now, expiry, ws);
      }
      r = __shfl_sync(kWarpAll, r, 0);  // also: lane 0 is done with the queue
      if (r != 0) {
        st = r > 0 ? kStInserted : kStBusy;
        break;
      }
    }
    if (lane == 0) {
      if (st == kStFull && retry) {
        retry[atomicAdd(retry_count, 1u)] = i;
      } else {
        if (st == kStBusy) latch_error(t, kErrLockTimeout);
        status[i] = st;
      }
    }
  }
}

template <int kBfsNodes>
__host__ __device__ constexpr size_t warp_search_bytes() {
  return kBfsNodes * sizeof(Node) + WarpSeen<kBfsNodes>::kSize * sizeof(uint32_t);
}

template <int kWarps, int kBfsNodes, int kBfsDepth>
__global__ void __launch_bounds__(kWarps * 32, 1) insert_phase2_warp(TableSet ts, const uint8_t* __restrict__ keys,
                                                                  const uint64_t* __restrict__ vals, uint32_t now,
                                                                  uint32_t expiry, uint8_t* __restrict__ status,
                                                                  Workspace ws, const uint32_t* list,
                                                                  const uint32_t* count_ptr, uint32_t* retry,
                                                                  uint32_t* retry_count, uint32_t max_keys) {
  pdl_wait();
  pdl_release();
  static_assert(kWarps * warp_search_bytes<kBfsNodes>() <= 48 * 1024, "search state exceeds 48 KB");
  __shared__ Node queues[kWarps][kBfsNodes];
  __shared__ uint32_t sets[kWarps][WarpSeen<kBfsNodes>::kSize];
  const uint32_t w = threadIdx.x >> 5;
  phase2_range_warp<kBfsNodes, kBfsDepth>(ts, keys, vals, now, expiry, status, ws, list, ld32_cg(count_ptr), retry,
                                          retry_count, max_keys, queues[w], sets[w], blockIdx.x * kWarps + w,
                                          gridDim.x * kWarps);
}

template <int kThreadsPerBlock, int kBfsNodes, int kBfsDepth>
__global__ void __launch_bounds__(kThreadsPerBlock) insert_phase2(TableSet ts, const uint8_t* __restrict__ keys,
                                                                  const uint64_t* __restrict__ vals, uint32_t now,
                                                                  uint32_t expiry, uint8_t* __restrict__ status,
                                                                  Workspace ws, const uint32_t* list,
                                                                  const uint32_t* count_ptr, uint32_t* retry,
                                                                  uint32_t* retry_count, uint32_t max_keys) {
  pdl_wait();
  pdl_release();
  static_assert(kThreadsPerBlock * kBfsNodes * sizeof(Node) <= 48 * 1024, "BFS state exceeds 48 KB");
  static_assert(kThreadsPerBlock % 32 == 0 &&
                    (kThreadsPerBlock / 32) * warp_search_bytes<kBfsNodes>() <= kBfsNodes * kThreadsPerBlock * sizeof(Node),
                "the warp form's state does not fit in the queues");
  __shared__ __align__(16) Node queues[kBfsNodes][kThreadsPerBlock];
  const uint32_t listed = ld32_cg(count_ptr);
  if (listed <= kGridWarpKeys) {
    // a short list: one warp per key, each warp's queue and visited set carved from the block's queues
    const uint32_t w = threadIdx.x >> 5;
    uint8_t* mine = reinterpret_cast<uint8_t*>(&queues[0][0]) + w * warp_search_bytes<kBfsNodes>();
    phase2_range_warp<kBfsNodes, kBfsDepth>(ts, keys, vals, now, expiry, status, ws, list, listed, retry,
                                            retry_count, max_keys, reinterpret_cast<Node*>(mine),
                                            reinterpret_cast<uint32_t*>(mine + kBfsNodes * sizeof(Node)),
                                            blockIdx.x * (kThreadsPerBlock / 32) + w,
                                            gridDim.x * (kThreadsPerBlock / 32));
    return;
  }
  const Queue q{&queues[0][threadIdx.x], kThreadsPerBlock};
  phase2_range<kBfsNodes, kBfsDepth>(ts, keys, vals, now, expiry, status, ws, list, listed, retry, retry_count,
                                     max_keys, q, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// ----------------------------------------------------- fixup and finish
// The two parts touch disjoint words (filters of the fixup list's buckets;
// status bytes of non-leader keys), so one launch runs both: every thread
// takes its share of the fixup list, and thread i < n finishes key i.
__device__ void fixup_finish_range(const TableSet& ts, uint64_t n, uint8_t* __restrict__ status, const Workspace& ws,
                                   uint64_t worker, uint64_t workers) {
  const uint64_t stride = workers;
  const uint64_t i = worker;
  if (ld32_cg(ws.counters + 2)) {  // the list overflowed: scan every bucket of every table
    for (uint32_t tb = 0; tb < ts.n_tables; ++tb) {
      const TableView t = ts.table(tb);
      for (uint64_t b = i; b < t.nb; b += stride)
        if (ld32_cg(moved_ptr(t, (uint32_t)b)) == 0u) st64_cg(bloom_ptr(t, (uint32_t)b), 0ull);
    }
  } else {
    const uint32_t count = min(ld32_cg(ws.counters + 1), ws.fix_cap);
    for (uint64_t j = i; j < count; j += stride) {
      const unsigned long long e = ws.fixup[j];
      const TableView t = ts.table((uint32_t)(e >> 32));
      const uint32_t b = (uint32_t)e;
      if (ld32_cg(moved_ptr(t, b)) == 0u) st64_cg(bloom_ptr(t, b), 0ull);
    }
  }
  for (uint64_t j = i; j < n; j += stride) {
    if (status[j] != kStFollower) continue;  // a leader: its outcome is final
    const uint32_t leader = ld32_cg(ws.first_at(ws.slot_of[j]));
    const uint8_t st = status[leader];
    status[j] = (st == kStInserted || st == kStUpdated) ? kStUpdated : st;  // FULL, BUSY, NO_TABLE copy through
  }
}

__global__ void __launch_bounds__(kThreads) insert_fixup_finish(TableSet ts, uint64_t n, uint8_t* __restrict__ status,
                                                                Workspace ws) {
  pdl_wait();
  pdl_release();
  fixup_finish_range(ts, n, status, ws, blockIdx.x * (uint64_t)blockDim.x + threadIdx.x,
                     (uint64_t)gridDim.x * blockDim.x);
}

// --------------------------------------------------- single-launch insert
// The whole insert call of a small batch in one cooperative launch: the
// stages of the chain above (dedup, phase 1, publication, the one-move pass,
// the three search passes, fixup and finish) run in order, separated by a
// grid barrier instead of kernel boundaries. A small batch spends most of a
// chain's time in the chain's nine dependent launches (each one's start and
// drain); here it pays two (the workspace clear and this kernel). All blocks
// are resident at once (cooperative launch, grid sized by the occupancy the
// kernel reaches), so the barrier cannot wait on a block that has not
// started. Search queues live in 48 KB of dynamic shared memory per block: the
// grid pass runs on 64 threads of every block (96 nodes each; on every warp
// for a short list), the second pass
// on every warp (192 nodes and a visited set each), the last on the first warp
// of every block (2048 nodes and the visited set).
constexpr int kSingleThreads = 256;
constexpr size_t kSingleSmem = 48 * 1024;
constexpr unsigned kSingleMinBlocks = 8;
// Bounded wait at a barrier: about 2-4 s of polls (each a load and a 64 ns sleep), longer than
// the bounded lock waits a stage may contain, so a barrier gives up only if a block never arrives.
constexpr int kBarrierSpins = 1 << 22;

static_assert(96 * 64 * sizeof(Node) <= kSingleSmem, "grid pass queues exceed the shared memory");
static_assert((kSingleThreads / 32) * warp_search_bytes<96>() <= kSingleSmem,
              "grid pass state (one warp per key) exceeds the shared memory");
static_assert((kSingleThreads / 32) * warp_search_bytes<192>() <= kSingleSmem,
              "second pass state exceeds the shared memory");
static_assert(warp_search_bytes<2048>() <= kSingleSmem, "last pass state exceeds the shared memory");

__device__ __forceinline__ uint32_t ld_acquire32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier over gridDim.x resident blocks. count and gen are two
// words of the workspace's zeroed counters: every block reads the generation,
// then arrives on the count; the last to arrive resets the count and advances
// the generation (release), and the others wait for it (acquire). Returns
// false if the wait gave up after kBarrierSpins polls.
__device__ bool grid_barrier(uint32_t* count, uint32_t* gen) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    asm volatile("fence.acq_rel.gpu;" ::: "memory");  // this block's writes before the arrival
    const uint32_t g = ld_acquire32(gen);
    if (atomicAdd(count, 1u) == gridDim.x - 1) {
      atomicExch(count, 0u);
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(gen) : "memory");
    } else {
      for (int spin = 0; ld_acquire32(gen) == g; ++spin) {
        if (spin >= kBarrierSpins) {
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");  // the other blocks' writes after it
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

__global__ void __launch_bounds__(kSingleThreads, 2) insert_single_launch(TableSet ts, const uint8_t* __restrict__ keys,
                                                                         const uint64_t* __restrict__ vals, uint64_t n,
                                                                         uint32_t now, uint32_t expiry,
                                                                         uint8_t* __restrict__ status, Workspace ws) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint32_t* bar_count = ws.counters + 8;
  uint32_t* bar_gen = ws.counters + 9;
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t threads = (uint64_t)gridDim.x * blockDim.x;
  bool ok = true;
  for (uint64_t i = tid; i < n; i += threads) dedup_one(keys, ts, ws, i);
  ok &= grid_barrier(bar_count, bar_gen);
  for (uint64_t i = tid; i < n; i += threads) phase1_one(ts, keys, vals, now, expiry, status, ws, i);
  ok &= grid_barrier(bar_count, bar_gen);
  for (uint64_t i = tid; i < n; i += threads) publish_one(ts, ws, i);
  ok &= grid_barrier(bar_count, bar_gen);
  // lists as in the chain: pending [0] -> one move -> retry [3] -> grid search -> pending [5] ->
  // second pass -> retry [6] -> last pass. A pass whose list is empty is skipped with its barrier;
  // every block reads the same count (final before the barrier), so all skip alike.
  if (ld32_cg(ws.counters + 0)) {
    move1_range(ts, keys, vals, now, expiry, status, ws, ws.pending, ws.counters + 0, ws.retry, ws.counters + 3,
                (uint32_t)tid, (uint32_t)threads);
    ok &= grid_barrier(bar_count, bar_gen);
  }
  Node* nodes = reinterpret_cast<Node*>(smem);
  const uint32_t w = threadIdx.x >> 5;
  if (const uint32_t listed = ld32_cg(ws.counters + 3)) {
    if (listed <= kGridWarpKeys) {  // a short list: one warp per key
      uint8_t* mine = smem + w * warp_search_bytes<96>();
      phase2_range_warp<96, 4>(ts, keys, vals, now, expiry, status, ws, ws.retry, listed, ws.pending,
                               ws.counters + 5, 0xFFFFFFFFu, reinterpret_cast<Node*>(mine),
                               reinterpret_cast<uint32_t*>(mine + 96 * sizeof(Node)),
                               blockIdx.x * (kSingleThreads / 32) + w, gridDim.x * (kSingleThreads / 32));
    } else if (threadIdx.x < 64) {
      const Queue q{nodes + threadIdx.x, 64};
      phase2_range<96, 4>(ts, keys, vals, now, expiry, status, ws, ws.retry, listed, ws.pending,
                          ws.counters + 5, 0xFFFFFFFFu, q, blockIdx.x * 64 + threadIdx.x, gridDim.x * 64);
    }
    ok &= grid_barrier(bar_count, bar_gen);
  }
  if (ld32_cg(ws.counters + 5)) {
    constexpr size_t kPer = warp_search_bytes<192>();
    uint8_t* mine = smem + w * kPer;
    phase2_range_warp<192, 5>(ts, keys, vals, now, expiry, status, ws, ws.pending, ld32_cg(ws.counters + 5), ws.retry,
                              ws.counters + 6, kSecondPassKeys, reinterpret_cast<Node*>(mine),
                              reinterpret_cast<uint32_t*>(mine + 192 * sizeof(Node)),
                              blockIdx.x * (kSingleThreads / 32) + w, gridDim.x * (kSingleThreads / 32));
    ok &= grid_barrier(bar_count, bar_gen);
  }
  if (ld32_cg(ws.counters + 6)) {
    if (w == 0)
      phase2_range_warp<2048, 6>(ts, keys, vals, now, expiry, status, ws, ws.retry, ld32_cg(ws.counters + 6),
                                 (uint32_t*)nullptr, (uint32_t*)nullptr, kLastPassKeys, nodes,
                                 reinterpret_cast<uint32_t*>(smem + 2048 * sizeof(Node)), blockIdx.x, gridDim.x);
    ok &= grid_barrier(bar_count, bar_gen);
  }
  fixup_finish_range(ts, n, status, ws, tid, threads);
  if (!ok && threadIdx.x == 0) latch_error(ts.table(0), kErrLockTimeout);
}

// ------------------------------------------------------- workspace reset
// The set's words alternate first (empty) and last (0), so each 16-byte
// vector holds two positions.
__global__ void __launch_bounds__(kThreads) workspace_clear(uint32_t* __restrict__ counters, uint32_t counter_words,
                                                            uint4* __restrict__ set, uint64_t n_vec,
                                                            uint4* __restrict__ dup, uint64_t dup_vec) {
  pdl_release();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (tid < counter_words) counters[tid] = 0u;
  for (uint64_t j = tid; j < n_vec; j += stride) set[j] = make_uint4(kEmpty, 0u, kEmpty, 0u);
  for (uint64_t j = tid; j < dup_vec; j += stride) dup[j] = make_uint4(0u, 0u, 0u, 0u);
}

__global__ void __launch_bounds__(kThreads) delete_kernel(TableSet ts, const uint8_t* __restrict__ keys, uint64_t n,
                                                          uint32_t now, uint8_t* __restrict__ status, Workspace ws) {
  pdl_wait();
  pdl_release();
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (!ts.valid(i)) {
    status[i] = kStNoTable;
    return;
  }
  uint32_t last;
  if (!is_leader(ws, i, last)) {
    status[i] = kStNotFound;
    return;
  }
  const TableView t = ts.of(i);
  const Key k = load_key(keys, i);
  const Addr a = address_of(k, t.nb, t.seed);
  uint64_t h[4];
  ld256_cg(bucket_ptr(t, a.b1), h);
  uint32_t b = a.b1;
  Snap s;
  s.w[0] = h[0];
  s.w[1] = h[1];
  int slot = find_key(t, b, (uint32_t)h[3], s, k, a.tag);
  if (slot < 0 && (h[2] & a.bits) == a.bits) {
    b = a.b2;
    ld256_cg(bucket_ptr(t, b), s.w);
    slot = find_key(t, b, (uint32_t)s.w[3], s, k, a.tag);
  }
  uint8_t st = kStNotFound;
  if (slot >= 0) {
    const bool was_alive = !t.timers || alive16(ld16_cg(expiry_ptr(t, b, slot)), now);
    const uint32_t old = atomicAnd(ctrl_ptr(t, b), ~((1u << slot) | (1u << (kInsecShift + slot))));
    // Sec. 4.1: removing a displaced key decrements its primary's counter; at
    // zero the filter is reset. No filter bit is set during a delete batch.
    if ((old >> (kInsecShift + slot)) & 1u) {
      if (atomicSub(moved_ptr(t, a.b1), 1u) == 1u)
        atomicExch(reinterpret_cast<unsigned long long*>(bloom_ptr(t, a.b1)), 0ull);
    }
    st = was_alive ? kStDeleted : kStNotFound;
  }
  status[i] = st;
}

unsigned grid_for(uint64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// Launch a kernel of an insert or delete call after its predecessor on the
// same stream, with programmatic stream serialization (see pdl_wait).
template <typename... Params, typename... Args>
cudaError_t launch_chained(void (*kernel)(Params...), unsigned grid, unsigned block, cudaStream_t s, Args... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace

cudaError_t launch_workspace_clear(const Workspace& ws, uint32_t counter_words, uint64_t n, cudaStream_t s) {
  // m is a power of two >= 64 and the set is 256-byte aligned: 2m words clear
  // as m / 2 whole 16-byte vectors; dup (256-byte aligned, its part of the
  // layout rounded up to 256 bytes) clears as ceil(n / 16) vectors
  const uint64_t n_vec = ((uint64_t)ws.m_mask + 1) / 2;
  const uint64_t dup_vec = (n + 15) / 16;
  uint64_t want = n_vec > counter_words ? n_vec : counter_words;
  want = want > dup_vec ? want : dup_vec;
  const uint64_t blocks = (want + kThreads - 1) / kThreads;
  const uint64_t cap = 16ull * device_sm_count();
  workspace_clear<<<(unsigned)(blocks < cap ? blocks : cap), kThreads, 0, s>>>(
      ws.counters, counter_words, reinterpret_cast<uint4*>(ws.set), n_vec, reinterpret_cast<uint4*>(ws.dup), dup_vec);
  return cudaGetLastError();
}

cudaError_t launch_dedup(const TableSet& ts, const uint8_t* keys, uint64_t n, const Workspace& ws, cudaStream_t s) {
  return launch_chained(dedup_kernel, grid_for(n, kThreads), kThreads, s, keys, n, ts, ws);
}

namespace {

std::atomic<int> g_insert_launch{kInsertLaunchChain};

// Blocks per SM the single-launch kernel reaches (queried once per device; 0 if
// it cannot run, or the device has too few SMs for its search passes).
int single_launch_blocks_per_sm() {
  constexpr int kMaxDevices = 64;
  static std::atomic<int> cache[kMaxDevices];  // 0 unknown, -1 cannot run, else blocks per SM
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return 0;
  }
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v) return v > 0 ? v : 0;
  int coop = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, insert_single_launch, kSingleThreads, kSingleSmem) !=
          cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  v = (coop && per_sm > 0 && (uint64_t)device_sm_count() * (per_sm < 2 ? per_sm : 2) >= kSingleMinBlocks)
          ? (per_sm < 2 ? per_sm : 2)
          : -1;
  cache[dev].store(v, std::memory_order_relaxed);
  return v > 0 ? v : 0;
}

cudaError_t launch_single(const TableSet& ts, const uint8_t* keys, const uint64_t* vals, uint64_t n, uint32_t now,
                          uint32_t expiry, uint8_t* status, const Workspace& ws, cudaStream_t s, int per_sm) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  // one thread per key up to the resident limit, and a few blocks for the warps of the search passes
  const uint64_t want = (n + kSingleThreads - 1) / kSingleThreads;
  const uint64_t lo = kSingleMinBlocks, hi = (uint64_t)device_sm_count() * per_sm;
  cfg.gridDim = dim3((unsigned)(want < lo ? lo : (want > hi ? hi : want)));
  cfg.blockDim = dim3(kSingleThreads);
  cfg.dynamicSmemBytes = kSingleSmem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, insert_single_launch, ts, keys, vals, n, now, expiry, status, ws);
}

}  // namespace

int set_insert_launch(int mode) {
  if (mode != kInsertLaunchChain && mode != kInsertLaunchSingle) return -1;
  return g_insert_launch.exchange(mode);
}

cudaError_t launch_insert(const TableSet& ts, const uint8_t* keys, const uint64_t* vals, uint64_t n, uint32_t now,
                          uint32_t expiry, uint8_t* status, const Workspace& ws, cudaStream_t s) {
  const int mode = g_insert_launch.load(std::memory_order_relaxed);
  if (mode == kInsertLaunchSingle) {
    const int per_sm = single_launch_blocks_per_sm();
    if (per_sm > 0) return launch_single(ts, keys, vals, n, now, expiry, status, ws, s, per_sm);
  }
  cudaError_t e = launch_dedup(ts, keys, n, ws, s);
  if (e != cudaSuccess) return e;
  e = launch_chained(insert_phase1, grid_for(n, kThreads), kThreads, s, ts, keys, vals, n, now, expiry, status, ws);
  if (e != cudaSuccess) return e;
  e = launch_chained(insert_publish, grid_for(n, kThreads), kThreads, s, ts, n, ws);
  if (e != cudaSuccess) return e;
  // lists: phase 1 -> pending [0] -> move1 -> retry [3] -> grid search ->
  // pending [5] -> second search -> retry [6] -> last search
  const unsigned sms = (unsigned)device_sm_count();
  e = launch_chained(insert_move1, sms * 16, kThreads, s, ts, keys, vals, now, expiry, status, ws,
                     (const uint32_t*)ws.pending, (const uint32_t*)(ws.counters + 0), ws.retry, ws.counters + 3);
  if (e != cudaSuccess) return e;
  e = launch_chained(insert_phase2<kP2Threads, 96, 4>, sms * 4, kP2Threads, s, ts, keys, vals, now, expiry, status,
                     ws, (const uint32_t*)ws.retry, (const uint32_t*)(ws.counters + 3), ws.pending, ws.counters + 5,
                     0xFFFFFFFFu);
  if (e != cudaSuccess) return e;
  // second pass, one warp per key: the keys the grid pass could not place
  e = launch_chained(insert_phase2_warp<8, 192, 5>, sms * 2, 8 * 32, s, ts, keys, vals, now, expiry, status, ws,
                     (const uint32_t*)ws.pending, (const uint32_t*)(ws.counters + 5), ws.retry, ws.counters + 6,
                     kSecondPassKeys);
  if (e != cudaSuccess) return e;
  // last pass, one warp per key: the widest search; a key is FULL only if it finds no path
  e = launch_chained(insert_phase2_warp<1, 2048, 6>, kLastPassKeys, 32, s, ts, keys, vals, now, expiry, status, ws,
                     (const uint32_t*)ws.retry, (const uint32_t*)(ws.counters + 6), (uint32_t*)nullptr,
                     (uint32_t*)nullptr, kLastPassKeys);
  if (e != cudaSuccess) return e;
  const unsigned fin_blocks = grid_for(n, kThreads);
  return launch_chained(insert_fixup_finish, fin_blocks > sms * 2 ? fin_blocks : sms * 2, kThreads, s, ts, n, status,
                        ws);
}

cudaError_t launch_delete(const TableSet& ts, const uint8_t* keys, uint64_t n, uint32_t now, uint8_t* status,
                          const Workspace& ws, cudaStream_t s) {
  cudaError_t e = launch_dedup(ts, keys, n, ws, s);
  if (e != cudaSuccess) return e;
  return launch_chained(delete_kernel, grid_for(n, kThreads), kThreads, s, ts, keys, n, now, status, ws);
}

}  // namespace ckpp
