// Batched insert-or-update (Sec. 2 cuckoo insertion; Sec. 4.1 filter and moved
// counter upkeep; Sec. 4.2 reuse of dead slots).
//
// Kernels, in stream order:
//   dedup   - groups equal keys of the batch in an open-addressing set in the
//             workspace: each key learns the lowest (leader) and highest batch
//             index of its group, which gives the batch the result of inserting
//             the keys one by one in index order.
//   phase1  - per leader: lock its two buckets, update in place if the key is
//             stored (alive or dead), else take the lowest free or dead slot of
//             the primary, else of the secondary; leaders with two full buckets
//             are queued for phase 2.
//   phase2  - per queued leader: breadth-first search for a cuckoo path without
//             locks, then execute it backwards, one move at a time, each under
//             the locks of its two buckets with the move re-validated; retry a
//             bounded number of times, else FULL.
//   fixup   - reset the filter of buckets whose moved counter reached zero off
//             their lock (the reset of Sec. 4.1, deferred so that it never races
//             a concurrent setter).
//   finish  - non-leader occurrences copy their leader's outcome (UPDATED, or
//             FULL/BUSY).
#include "mutate.cuh"

namespace ckpp {

namespace {

constexpr int kThreads = 256;
constexpr int kBfsNodes = 128;
constexpr int kBfsDepth = 4;
constexpr int kPathAttempts = 8;

__device__ __forceinline__ Key load_key(const uint8_t* keys, uint64_t i) {
  uint64_t a, b;
  asm volatile("ld.global.nc.v2.u64 {%0,%1}, [%2];" : "=l"(a), "=l"(b) : "l"(keys + 16 * i));
  return Key{a, b};
}

// ---------------------------------------------------------------- dedup
__global__ void __launch_bounds__(kThreads) dedup_kernel(const uint8_t* __restrict__ keys, uint64_t n, uint64_t seed,
                                                         Workspace ws) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Key k = load_key(keys, i);
  uint32_t pos = (uint32_t)(hash_key(k, seed) >> 16) & ws.m_mask;
  for (uint32_t probe = 0; probe <= ws.m_mask; ++probe) {
    uint32_t cur = ld32_cg(ws.set_first + pos);
    if (cur == kEmpty) {
      cur = atomicCAS(ws.set_first + pos, kEmpty, (uint32_t)i);
      if (cur == kEmpty) {
        atomicMax(ws.set_last + pos, (uint32_t)i);
        ws.slot_of[i] = pos;
        return;
      }
    }
    // set_first only ever holds batch indices of one key group, so the key at
    // index cur is that group's key even while atomicMin lowers cur.
    const Key o = load_key(keys, cur);
    if (o.k0 == k.k0 && o.k1 == k.k1) {
      atomicMin(ws.set_first + pos, (uint32_t)i);
      atomicMax(ws.set_last + pos, (uint32_t)i);
      ws.slot_of[i] = pos;
      return;
    }
    pos = (pos + 1) & ws.m_mask;
  }
}

__device__ __forceinline__ bool is_leader(const Workspace& ws, uint64_t i, uint32_t& last) {
  const uint32_t pos = ws.slot_of[i];
  if (ws.set_first[pos] != (uint32_t)i) return false;
  last = ws.set_last[pos];
  return true;
}

// --------------------------------------------------------------- phase 1
__global__ void __launch_bounds__(kThreads) insert_phase1(TableView t, const uint8_t* __restrict__ keys,
                                                          const uint64_t* __restrict__ vals, uint64_t n,
                                                          uint32_t now, uint32_t expiry, uint8_t* __restrict__ status,
                                                          Workspace ws) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t last;
  if (!is_leader(ws, i, last)) return;
  const uint64_t v = vals[last];
  const Key k = load_key(keys, i);
  const Addr a = address_of(k, t.nb, t.seed);
  uint32_t c1, c2;
  if (!lock_pair(t, a.b1, a.b2, c1, c2)) {
    status[i] = kStBusy;
    latch_error(t, kErrLockTimeout);
    return;
  }
  Snap s1, s2;
  snap_bucket(t, a.b1, s1);
  snap_bucket(t, a.b2, s2);
  uint8_t st = 0;
  // Upsert: a stored copy of the key (alive or dead) is updated in place.
  uint32_t b = a.b1;
  const Snap* sb = &s1;
  int slot = find_key(t, a.b1, c1, s1, k, a.tag);
  if (slot < 0) {
    b = a.b2;
    sb = &s2;
    slot = find_key(t, a.b2, c2, s2, k, a.tag);
  }
  if (slot >= 0) {
    const bool was_alive = !t.timers || alive16(snap_expiry(*sb, slot), now);
    st64_cg(record_ptr(t, b, slot) + 16, v);
    if (t.timers) st16_cg(expiry_ptr(t, b, slot), expiry);
    st = was_alive ? kStUpdated : kStInserted;
  } else {
    const uint32_t f1 = free_mask(t, c1, s1, now);
    const uint32_t f2 = f1 ? 0u : free_mask(t, c2, s2, now);
    if (f1 || f2) {
      b = f1 ? a.b1 : a.b2;
      uint32_t& cb = f1 ? c1 : c2;
      slot = __ffs(f1 ? f1 : f2) - 1;
      if ((cb >> slot) & 1u) evict_entry(t, b, slot, cb, ws);
      place_entry(t, b, slot, k, v, a, expiry, cb);
      st = kStInserted;
    } else {
      ws.pending[atomicAdd(ws.counters + 0, 1u)] = (uint32_t)i;
    }
  }
  unlock_pair(t, a.b1, a.b2, c1, c2);
  if (st) status[i] = st;
}

// --------------------------------------------------------------- phase 2
struct Node {
  uint32_t bucket;
  int16_t parent;
  uint8_t slot;   // slot of the parent bucket whose entry moves into this bucket
  uint8_t depth;
};

// Place k into the lowest free or dead slot of its primary, else secondary.
// 1 placed, 0 no room, -1 lock timeout.
__device__ int try_place(const TableView& t, const Key& k, uint64_t v, const Addr& a, uint32_t now, uint32_t expiry,
                         const Workspace& ws) {
  uint32_t c1, c2;
  if (!lock_pair(t, a.b1, a.b2, c1, c2)) return -1;
  Snap s1, s2;
  snap_bucket(t, a.b1, s1);
  snap_bucket(t, a.b2, s2);
  const uint32_t f1 = free_mask(t, c1, s1, now);
  const uint32_t f2 = f1 ? 0u : free_mask(t, c2, s2, now);
  int placed = 0;
  if (f1 || f2) {
    const uint32_t b = f1 ? a.b1 : a.b2;
    uint32_t& cb = f1 ? c1 : c2;
    const uint32_t slot = __ffs(f1 ? f1 : f2) - 1;
    if ((cb >> slot) & 1u) evict_entry(t, b, slot, cb, ws);
    place_entry(t, b, slot, k, v, a, expiry, cb);
    placed = 1;
  }
  unlock_pair(t, a.b1, a.b2, c1, c2);
  return placed;
}

// Breadth-first search over buckets from b1 and b2 (lock-free reads; the moves
// re-validate). Returns the index of a node whose bucket has a free or dead
// slot (in hole), or -1.
__device__ int bfs(const TableView& t, const Addr& a, uint32_t now, Node* q, uint32_t& hole) {
  int nq = 0;
  q[nq++] = Node{a.b1, -1, 0, 0};
  q[nq++] = Node{a.b2, -1, 0, 0};
  for (int qi = 0; qi < nq; ++qi) {
    Snap s;
    snap_bucket(t, q[qi].bucket, s);
    const uint32_t ctrl = (uint32_t)s.w[3];
    const uint32_t f = free_mask(t, ctrl, s, now);
    if (f) {
      hole = __ffs(f) - 1;
      return qi;
    }
    if (q[qi].depth >= kBfsDepth) continue;
    for (uint32_t sl = 0; sl < kSlots && nq < kBfsNodes; ++sl) {
      uint64_t r[4];
      ld256_cg(record_ptr(t, q[qi].bucket, sl), r);
      const Addr e = address_of(Key{r[0], r[1]}, t.nb, t.seed);
      const uint32_t y = (e.b1 == q[qi].bucket) ? e.b2 : e.b1;
      bool seen = false;
      for (int j = 0; j < nq; ++j) seen |= (q[j].bucket == y);
      if (!seen) q[nq++] = Node{y, (int16_t)qi, (uint8_t)sl, (uint8_t)(q[qi].depth + 1)};
    }
  }
  return -1;
}

// Move the entry in slot sx of bucket x to free (or dead) slot sy of its other
// bucket y, under both locks, after re-validating both. Sec. 4.1: a move from
// the primary to the secondary sets the entry's bits in the primary's filter
// and increments its counter; the reverse move decrements the counter and
// resets the filter at zero. 1 moved, 0 stale path, -1 lock timeout.
__device__ int move_entry(const TableView& t, uint32_t x, uint32_t sx, uint32_t y, uint32_t sy, uint32_t now,
                          const Workspace& ws) {
  uint32_t cx, cy;
  if (!lock_pair(t, x, y, cx, cy)) return -1;
  int ok = 0;
  if ((cx >> sx) & 1u) {
    uint64_t r[4];
    ld256_cg(record_ptr(t, x, sx), r);
    const Addr e = address_of(Key{r[0], r[1]}, t.nb, t.seed);
    const bool from_primary = (e.b1 == x);
    const bool valid_src = from_primary ? (e.b2 == y) : (e.b2 == x && e.b1 == y);
    bool dst_free = !((cy >> sy) & 1u);
    uint32_t dst_exp = 0;
    if (!dst_free && t.timers) {
      dst_exp = ld16_cg(expiry_ptr(t, y, sy));
      dst_free = !alive16(dst_exp, now);
    }
    if (valid_src && dst_free) {
      if ((cy >> sy) & 1u) evict_entry(t, y, sy, cy, ws);
      st256_cg(record_ptr(t, y, sy), r[0], r[1], r[2], r[3]);
      st16_cg(tag_ptr(t, y, sy), e.tag);
      if (t.timers) st16_cg(expiry_ptr(t, y, sy), ld16_cg(expiry_ptr(t, x, sx)));
      cy |= 1u << sy;
      if (from_primary) {
        cy |= 1u << (kInsecShift + sy);
        atomicOr(reinterpret_cast<unsigned long long*>(bloom_ptr(t, x)), (unsigned long long)e.bits);
        atomicAdd(moved_ptr(t, x), 1u);
      } else {
        cy &= ~(1u << (kInsecShift + sy));
        if (atomicSub(moved_ptr(t, y), 1u) == 1u) {
          atomicExch(reinterpret_cast<unsigned long long*>(bloom_ptr(t, y)), 0ull);
        }
      }
      cx &= ~((1u << sx) | (1u << (kInsecShift + sx)));
      ok = 1;
    }
  }
  unlock_pair(t, x, y, cx, cy);
  return ok;
}

__global__ void __launch_bounds__(128) insert_phase2(TableView t, const uint8_t* __restrict__ keys,
                                                     const uint64_t* __restrict__ vals, uint32_t now, uint32_t expiry,
                                                     uint8_t* __restrict__ status, Workspace ws) {
  const uint32_t count = ld32_cg(ws.counters + 0);
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < count; j += gridDim.x * blockDim.x) {
    const uint32_t i = ws.pending[j];
    const uint64_t v = vals[ws.set_last[ws.slot_of[i]]];
    const Key k = load_key(keys, i);
    const Addr a = address_of(k, t.nb, t.seed);
    uint8_t st = kStFull;
    Node q[kBfsNodes];
    for (int attempt = 0; attempt < kPathAttempts; ++attempt) {
      const int placed = try_place(t, k, v, a, now, expiry, ws);
      if (placed != 0) {
        st = placed > 0 ? kStInserted : kStBusy;
        break;
      }
      uint32_t hole = 0;
      int node = bfs(t, a, now, q, hole);
      if (node < 0) break;  // no cuckoo path within the search bound: FULL
      // Execute the path backwards: each entry moves into the hole ahead of it.
      int r = 1;
      while (q[node].parent >= 0 && r > 0) {
        const int par = q[node].parent;
        r = move_entry(t, q[par].bucket, q[node].slot, q[node].bucket, hole, now, ws);
        hole = q[node].slot;
        node = par;
      }
      if (r < 0) {
        st = kStBusy;
        break;
      }
    }
    if (st == kStBusy) latch_error(t, kErrLockTimeout);
    status[i] = st;
  }
}

// ----------------------------------------------------- fixup and finish
__global__ void bloom_fixup(TableView t, Workspace ws) {
  const uint32_t stride = gridDim.x * blockDim.x;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (ld32_cg(ws.counters + 2)) {
    for (uint64_t b = tid; b < t.nb; b += stride)
      if (ld32_cg(moved_ptr(t, (uint32_t)b)) == 0u) st64_cg(bloom_ptr(t, (uint32_t)b), 0ull);
  } else {
    const uint32_t count = min(ld32_cg(ws.counters + 1), ws.fix_cap);
    for (uint32_t j = tid; j < count; j += stride) {
      const uint32_t b = ws.fixup[j];
      if (ld32_cg(moved_ptr(t, b)) == 0u) st64_cg(bloom_ptr(t, b), 0ull);
    }
  }
}

__global__ void __launch_bounds__(kThreads) insert_finish(uint64_t n, uint8_t* __restrict__ status, Workspace ws) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t leader = ws.set_first[ws.slot_of[i]];
  if (leader == (uint32_t)i) return;
  const uint8_t st = status[leader];
  status[i] = (st == kStInserted || st == kStUpdated) ? kStUpdated : st;
}

__global__ void __launch_bounds__(kThreads) delete_kernel(TableView t, const uint8_t* __restrict__ keys, uint64_t n,
                                                          uint32_t now, uint8_t* __restrict__ status, Workspace ws) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t last;
  if (!is_leader(ws, i, last)) {
    status[i] = kStNotFound;
    return;
  }
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

}  // namespace

cudaError_t launch_dedup(const TableView& t, const uint8_t* keys, uint64_t n, const Workspace& ws, cudaStream_t s) {
  dedup_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(keys, n, t.seed, ws);
  return cudaGetLastError();
}

cudaError_t launch_insert(const TableView& t, const uint8_t* keys, const uint64_t* vals, uint64_t n, uint32_t now,
                          uint32_t expiry, uint8_t* status, const Workspace& ws, cudaStream_t s) {
  cudaError_t e = launch_dedup(t, keys, n, ws, s);
  if (e != cudaSuccess) return e;
  insert_phase1<<<grid_for(n, kThreads), kThreads, 0, s>>>(t, keys, vals, n, now, expiry, status, ws);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const unsigned p2_blocks = (unsigned)std::min<uint64_t>(grid_for(n, 128), 152 * 4);
  insert_phase2<<<p2_blocks, 128, 0, s>>>(t, keys, vals, now, expiry, status, ws);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  bloom_fixup<<<152 * 2, 256, 0, s>>>(t, ws);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  insert_finish<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, status, ws);
  return cudaGetLastError();
}

cudaError_t launch_delete(const TableView& t, const uint8_t* keys, uint64_t n, uint32_t now, uint8_t* status,
                          const Workspace& ws, cudaStream_t s) {
  cudaError_t e = launch_dedup(t, keys, n, ws, s);
  if (e != cudaSuccess) return e;
  delete_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(t, keys, n, now, status, ws);
  return cudaGetLastError();
}

}  // namespace ckpp
