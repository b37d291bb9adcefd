// Internal to libckpp.so: the host-side table handle and the argument and
// workspace helpers shared by the C ABI implementation files.
#pragma once

#include <cstdint>
#include <cstring>

#include "../../include/ckpp.h"
#include "ckpp_kernels.h"

struct ckpp_table {
  ckpp_geometry geo;
  uint8_t* base;
  size_t bytes;
  ckpp::TableView view;
  int have_epoch;
  uint32_t last_scan;
};

namespace ckpp {
namespace api {

constexpr size_t kAlign = 256;

constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

inline bool geometry_ok(const ckpp_geometry* g) {
  return g && g->n_buckets >= 2 && g->n_buckets <= 0xFFFFFFFFull && g->slots_per_bucket == kSlots &&
         (g->flags & ~CKPP_TIMERS) == 0;
}

inline size_t table_bytes(const ckpp_geometry* g) { return kHeaderBytes + (size_t)g->n_buckets * kBucketBytes; }

// Workspace of an n-key batch: counters | set[2m] (first and last index per
// position, interleaved) | slot_of[n] | dup[n] (bytes) | pending[n] | retry[n]
// | claim[n] (8 bytes each) | fixup[fix_cap] (8 bytes each), each part
// 256-byte aligned.
struct WsLayout {
  uint64_t m = 0;
  uint32_t fix_cap = 0;
  size_t off_set = 0, off_slot = 0, off_dup = 0, off_pending = 0, off_retry = 0, off_claim = 0, off_fixup = 0,
         total = 0;
};

constexpr WsLayout ws_layout(uint64_t n) {
  WsLayout L;
  // The dedup set probes linearly, and its longest probe sequence (a dependent
  // key read and CAS per step) sets the dedup kernel's time: at load 1/2 about
  // 30 steps for 32K keys, at 1/8 about 7. So m is a power of two of at least
  // 8n up to 2^17 keys (at most 8 MB of set) and 4n above (at most 2^32).
  uint64_t m = 64;
  const uint64_t want = n <= (1ull << 17) ? 8 * n : 4 * n;
  while (m < want) m <<= 1;
  L.m = m;
  L.fix_cap = (uint32_t)(n < (1ull << 22) ? n : (1ull << 22)) + 64;
  size_t off = kAlign;  // counters
  L.off_set = off;
  off = align_up(off + 8 * m, kAlign);
  L.off_slot = off;
  off = align_up(off + 4 * n, kAlign);
  L.off_dup = off;
  off = align_up(off + n, kAlign);
  L.off_pending = off;
  off = align_up(off + 4 * n, kAlign);
  L.off_retry = off;
  off = align_up(off + 4 * n, kAlign);
  L.off_claim = off;
  off = align_up(off + 8 * n, kAlign);
  L.off_fixup = off;
  off = align_up(off + 8 * (size_t)L.fix_cap, kAlign);
  L.total = off;
  return L;
}

inline int prepare_workspace(uint64_t n, void* workspace, size_t bytes, cudaStream_t s, Workspace& ws) {
  const WsLayout L = ws_layout(n);
  if (!workspace || bytes < L.total || !aligned(workspace, kAlign)) return CKPP_EINVAL;
  uint8_t* w = static_cast<uint8_t*>(workspace);
  ws.counters = reinterpret_cast<uint32_t*>(w);
  ws.set = reinterpret_cast<uint32_t*>(w + L.off_set);
  ws.slot_of = reinterpret_cast<uint32_t*>(w + L.off_slot);
  ws.dup = w + L.off_dup;
  ws.pending = reinterpret_cast<uint32_t*>(w + L.off_pending);
  ws.retry = reinterpret_cast<uint32_t*>(w + L.off_retry);
  ws.claim = reinterpret_cast<unsigned long long*>(w + L.off_claim);
  ws.fixup = reinterpret_cast<unsigned long long*>(w + L.off_fixup);
  ws.m_mask = (uint32_t)(L.m - 1);
  ws.fix_cap = L.fix_cap;
  return launch_workspace_clear(ws, (uint32_t)(kAlign / 4), n, s) == cudaSuccess ? CKPP_OK : CKPP_ECUDA;
}

// Sec. 4.2: a timed call more than 64512 units after the last scan could see
// expired 16-bit timers wrap around and revive.
inline int time_check(ckpp_table* t, uint32_t now) {
  if (!(t->geo.flags & CKPP_TIMERS)) return CKPP_OK;
  if (!t->have_epoch) {
    t->have_epoch = 1;
    t->last_scan = now;
  }
  return (uint32_t)(now - t->last_scan) > kMaxStale ? CKPP_ESTALE : CKPP_OK;
}

inline int cuda_rc(cudaError_t e) { return e == cudaSuccess ? CKPP_OK : CKPP_ECUDA; }

// Where a buffer lives: 0 device (or managed), 1 pinned host memory mapped
// into the device's address space, -1 not reachable by the device.
inline int residency(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return 0;
  if (a.type == cudaMemoryTypeHost && a.devicePointer == p) return 1;
  return -1;
}

// One table as a TableSet.
inline TableSet one_table(const ckpp_table* t) { return TableSet{t->view, nullptr, nullptr, 1u}; }

inline int check_keys(const ckpp_key* keys, uint64_t n) {
  if (n > kMaxBatch) return CKPP_EINVAL;
  if (n && (!keys || !aligned(keys, 16))) return CKPP_EINVAL;
  return CKPP_OK;
}

}  // namespace api
}  // namespace ckpp
