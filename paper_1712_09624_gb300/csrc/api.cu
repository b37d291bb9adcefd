// C ABI of libckpp.so (declared in include/ckpp.h): argument checks, the
// host-side table handle, workspace carving and kernel dispatch. No call here
// allocates device memory; every device buffer belongs to the caller.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>

#include "../../include/ckpp.h"
#include "ckpp_kernels.h"

using namespace ckpp;

struct ckpp_table {
  ckpp_geometry geo;
  uint8_t* base;
  size_t bytes;
  TableView view;
  int have_epoch;
  uint32_t last_scan;
};

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

bool geometry_ok(const ckpp_geometry* g) {
  return g && g->n_buckets >= 2 && g->n_buckets <= 0xFFFFFFFFull && g->slots_per_bucket == kSlots &&
         (g->flags & ~CKPP_TIMERS) == 0;
}

uint32_t bucket_shift(const ckpp_geometry* g) { return (g->flags & CKPP_TIMERS) ? 6u : 5u; }

size_t table_bytes(const ckpp_geometry* g) {
  return kHeaderBytes + (size_t)g->n_buckets * ((size_t)1 << bucket_shift(g)) +
         (size_t)g->n_buckets * kSlots * kRecordBytes;
}

// Workspace of an n-key batch: counters | set_first[m] | set_last[m] |
// slot_of[n] | pending[n] | fixup[fix_cap], each part 256-byte aligned.
struct WsLayout {
  uint64_t m;
  uint32_t fix_cap;
  size_t off_first, off_last, off_slot, off_pending, off_fixup, total;
};

WsLayout ws_layout(uint64_t n) {
  WsLayout L;
  uint64_t m = 64;
  while (m < 2 * n) m <<= 1;
  L.m = m;
  L.fix_cap = (uint32_t)std::min<uint64_t>(n, 1ull << 22) + 64;
  size_t off = kAlign;  // counters
  L.off_first = off;
  off = align_up(off + 4 * m, kAlign);
  L.off_last = off;
  off = align_up(off + 4 * m, kAlign);
  L.off_slot = off;
  off = align_up(off + 4 * n, kAlign);
  L.off_pending = off;
  off = align_up(off + 4 * n, kAlign);
  L.off_fixup = off;
  off = align_up(off + 4 * (size_t)L.fix_cap, kAlign);
  L.total = off;
  return L;
}

int prepare_workspace(uint64_t n, void* workspace, size_t bytes, cudaStream_t s, Workspace& ws) {
  const WsLayout L = ws_layout(n);
  if (!workspace || bytes < L.total || !aligned(workspace, kAlign)) return CKPP_EINVAL;
  uint8_t* w = static_cast<uint8_t*>(workspace);
  ws.counters = reinterpret_cast<uint32_t*>(w);
  ws.set_first = reinterpret_cast<uint32_t*>(w + L.off_first);
  ws.set_last = reinterpret_cast<uint32_t*>(w + L.off_last);
  ws.slot_of = reinterpret_cast<uint32_t*>(w + L.off_slot);
  ws.pending = reinterpret_cast<uint32_t*>(w + L.off_pending);
  ws.fixup = reinterpret_cast<uint32_t*>(w + L.off_fixup);
  ws.m_mask = (uint32_t)(L.m - 1);
  ws.fix_cap = L.fix_cap;
  if (cudaMemsetAsync(w, 0, kAlign, s) != cudaSuccess) return CKPP_ECUDA;
  if (cudaMemsetAsync(ws.set_first, 0xFF, 4 * L.m, s) != cudaSuccess) return CKPP_ECUDA;
  if (cudaMemsetAsync(ws.set_last, 0, 4 * L.m, s) != cudaSuccess) return CKPP_ECUDA;
  return CKPP_OK;
}

// Sec. 4.2: a timed call more than 64512 units after the last scan could see
// expired 16-bit timers wrap around and revive.
int time_check(ckpp_table* t, uint32_t now) {
  if (!(t->geo.flags & CKPP_TIMERS)) return CKPP_OK;
  if (!t->have_epoch) {
    t->have_epoch = 1;
    t->last_scan = now;
  }
  return (uint32_t)(now - t->last_scan) > kMaxStale ? CKPP_ESTALE : CKPP_OK;
}

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? CKPP_OK : CKPP_ECUDA; }

// Where a buffer lives: 0 device (or managed), 1 pinned host memory mapped
// into the device's address space, -1 not reachable by the device.
int residency(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return 0;
  if (a.type == cudaMemoryTypeHost && a.devicePointer == p) return 1;
  return -1;
}

int check_keys(const ckpp_key* keys, uint64_t n) {
  if (n > kMaxBatch) return CKPP_EINVAL;
  if (n && (!keys || !aligned(keys, 16))) return CKPP_EINVAL;
  return CKPP_OK;
}

}  // namespace

extern "C" {

size_t ckpp_required_bytes(const ckpp_geometry* geometry) {
  return geometry_ok(geometry) ? table_bytes(geometry) : 0;
}

size_t ckpp_workspace_bytes(uint64_t n) { return n > kMaxBatch ? 0 : ws_layout(n).total; }

int ckpp_create(ckpp_table** out, const ckpp_geometry* geometry, void* dev_buf, size_t bytes, ckpp_stream_t stream) {
  if (!out || !geometry_ok(geometry) || !dev_buf || !aligned(dev_buf, kAlign) || bytes < table_bytes(geometry))
    return CKPP_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  ckpp_table* t = new (std::nothrow) ckpp_table;
  if (!t) return CKPP_EINVAL;
  std::memset(t, 0, sizeof *t);
  t->geo = *geometry;
  t->base = static_cast<uint8_t*>(dev_buf);
  t->bytes = table_bytes(geometry);
  t->view.buckets = t->base + kHeaderBytes;
  t->view.records = t->view.buckets + (size_t)geometry->n_buckets * ((size_t)1 << bucket_shift(geometry));
  t->view.err = reinterpret_cast<uint32_t*>(t->base + kHdrErr);
  t->view.nb = geometry->n_buckets;
  t->view.seed = geometry->seed;
  t->view.bucket_shift = bucket_shift(geometry);
  t->view.timers = (geometry->flags & CKPP_TIMERS) ? 1u : 0u;
  if (cudaMemsetAsync(t->base, 0, t->bytes, s) != cudaSuccess ||
      launch_init_header(t->base, geometry->n_buckets, geometry->slots_per_bucket, geometry->flags, geometry->seed,
                         s) != cudaSuccess) {
    delete t;
    return CKPP_ECUDA;
  }
  *out = t;
  return CKPP_OK;
}

int ckpp_destroy(ckpp_table* table) {
  if (!table) return CKPP_EINVAL;
  delete table;
  return CKPP_OK;
}

int ckpp_bulk_lookup(ckpp_table* t, const ckpp_key* keys, uint64_t n, uint64_t* out_vals, uint8_t* out_found,
                     uint32_t now, uint16_t refresh_ttl, ckpp_stream_t stream) {
  if (!t || check_keys(keys, n) || refresh_ttl >= kAliveWindow) return CKPP_EINVAL;
  if (n && (!out_vals || !out_found || !aligned(out_vals, 8))) return CKPP_EINVAL;
  if (int rc = time_check(t, now)) return rc;
  if (!n) return CKPP_OK;
  const int rk = residency(keys), rv = residency(out_vals), rf = residency(out_found);
  if (rk < 0 || rv < 0 || rf < 0) return CKPP_EINVAL;
  const bool host_io = rk == 1 || rv == 1 || rf == 1;
  return cuda_rc(launch_lookup(t->view, reinterpret_cast<const uint8_t*>(keys), n, out_vals, out_found, now,
                               refresh_ttl, host_io, reinterpret_cast<cudaStream_t>(stream)));
}

int ckpp_bulk_insert(ckpp_table* t, const ckpp_key* keys, const uint64_t* vals, uint64_t n, uint32_t now,
                     uint16_t ttl, uint8_t* status, void* workspace, size_t workspace_bytes, ckpp_stream_t stream) {
  if (!t || check_keys(keys, n) || ttl >= kAliveWindow) return CKPP_EINVAL;
  if (n && (!vals || !status || !aligned(vals, 8))) return CKPP_EINVAL;
  if (int rc = time_check(t, now)) return rc;
  if (!n) return CKPP_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Workspace ws;
  if (int rc = prepare_workspace(n, workspace, workspace_bytes, s, ws)) return rc;
  return cuda_rc(launch_insert(t->view, reinterpret_cast<const uint8_t*>(keys), vals, n, now,
                               (now + ttl) & 0xFFFFu, status, ws, s));
}

int ckpp_bulk_delete(ckpp_table* t, const ckpp_key* keys, uint64_t n, uint32_t now, uint8_t* status,
                     void* workspace, size_t workspace_bytes, ckpp_stream_t stream) {
  if (!t || check_keys(keys, n)) return CKPP_EINVAL;
  if (n && !status) return CKPP_EINVAL;
  if (int rc = time_check(t, now)) return rc;
  if (!n) return CKPP_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Workspace ws;
  if (int rc = prepare_workspace(n, workspace, workspace_bytes, s, ws)) return rc;
  return cuda_rc(launch_delete(t->view, reinterpret_cast<const uint8_t*>(keys), n, now, status, ws, s));
}

int ckpp_expire(ckpp_table* t, uint32_t now, uint64_t* d_n_expired, ckpp_stream_t stream) {
  if (!t || (d_n_expired && !aligned(d_n_expired, 8))) return CKPP_EINVAL;
  t->have_epoch = 1;
  t->last_scan = now;
  if (!t->view.timers) return CKPP_OK;
  return cuda_rc(launch_expire(t->view, now, reinterpret_cast<unsigned long long*>(d_n_expired),
                               reinterpret_cast<cudaStream_t>(stream)));
}

int ckpp_stats_get(ckpp_table* t, uint32_t now, ckpp_stats* out, ckpp_stream_t stream) {
  if (!t || !out) return CKPP_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // Device accumulators live in the header's spare bytes 64..247 (23 x u64).
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(t->base + 64);
  unsigned long long host[23];
  if (cudaMemsetAsync(acc, 0, sizeof host, s) != cudaSuccess) return CKPP_ECUDA;
  if (launch_stats(t->view, now, acc, s) != cudaSuccess) return CKPP_ECUDA;
  if (cudaMemcpyAsync(host, acc, sizeof host, cudaMemcpyDeviceToHost, s) != cudaSuccess) return CKPP_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CKPP_ECUDA;
  std::memset(out, 0, sizeof *out);
  out->n_buckets = t->geo.n_buckets;
  out->n_slots = t->geo.n_buckets * kSlots;
  out->n_occupied = host[0];
  out->n_live = host[1];
  out->n_in_secondary = host[2];
  out->n_moved_zero = host[3];
  out->moved_sum = host[4];
  out->bloom_bits_set = host[5];
  out->bloom_pop_sq = host[6];
  for (int j = 0; j < 16; ++j) out->moved_hist[j] = host[7 + j];
  return CKPP_OK;
}

int ckpp_lookup_probe_counts(ckpp_table* t, const ckpp_key* keys, uint64_t n, uint32_t now, uint64_t* d_counts,
                             ckpp_stream_t stream) {
  if (!t || check_keys(keys, n) || !d_counts || !aligned(d_counts, 8)) return CKPP_EINVAL;
  if (int rc = time_check(t, now)) return rc;
  if (!n) return CKPP_OK;
  return cuda_rc(launch_probe_counts(t->view, reinterpret_cast<const uint8_t*>(keys), n, now,
                                     reinterpret_cast<unsigned long long*>(d_counts),
                                     reinterpret_cast<cudaStream_t>(stream)));
}

int ckpp_sync_status(ckpp_table* t, ckpp_stream_t stream) {
  if (!t) return CKPP_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint32_t err = 0;
  if (cudaMemcpyAsync(&err, t->view.err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return CKPP_ECUDA;
  if (cudaMemsetAsync(t->view.err, 0, 4, s) != cudaSuccess) return CKPP_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CKPP_ECUDA;
  return err ? CKPP_EBUSY : CKPP_OK;
}

int ckpp_get_geometry(const ckpp_table* t, ckpp_geometry* out) {
  if (!t || !out) return CKPP_EINVAL;
  *out = t->geo;
  return CKPP_OK;
}

int ckpp_get_last_scan(const ckpp_table* t, uint32_t* last_scan, int* have_epoch) {
  if (!t || !last_scan || !have_epoch) return CKPP_EINVAL;
  *last_scan = t->last_scan;
  *have_epoch = t->have_epoch;
  return CKPP_OK;
}

const char* ckpp_error_string(int code) {
  switch (code) {
    case CKPP_OK: return "ok";
    case CKPP_EINVAL: return "invalid argument";
    case CKPP_ECUDA: return "CUDA error";
    case CKPP_ESTALE: return "more than 64512 time units since the last expire scan";
    case CKPP_EBUSY: return "a bounded device wait gave up";
    default: return "unknown error";
  }
}

int ckpp_abi_version(void) { return CKPP_ABI_VERSION; }

}  // extern "C"
