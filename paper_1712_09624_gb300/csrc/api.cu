// C ABI of libckpp.so (declared in include/ckpp.h): argument checks, the
// host-side table handle, workspace carving and kernel dispatch. No call here
// allocates device memory; every device buffer belongs to the caller.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "api_internal.h"

using namespace ckpp;
using namespace ckpp::api;

static_assert(kAbiVersion == CKPP_ABI_VERSION, "device and C ABI versions differ");


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
  t->view.err = reinterpret_cast<uint32_t*>(t->base + kHdrErr);
  t->view.nb = geometry->n_buckets;
  t->view.seed = geometry->seed;
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

int ckpp_attach(ckpp_table** out, void* dev_buf, size_t bytes, uint32_t now, ckpp_stream_t stream) {
  if (!out || !dev_buf || !aligned(dev_buf, kAlign) || bytes < kHeaderBytes) return CKPP_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint8_t hdr[kHeaderBytes];
  if (cudaMemcpyAsync(hdr, dev_buf, kHeaderBytes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return CKPP_ECUDA;
  uint32_t magic, abi, slots, flags;
  uint64_t nb, seed;
  std::memcpy(&magic, hdr + kHdrMagic, 4);
  std::memcpy(&abi, hdr + kHdrAbi, 4);
  std::memcpy(&nb, hdr + kHdrBuckets, 8);
  std::memcpy(&slots, hdr + kHdrSlots, 4);
  std::memcpy(&flags, hdr + kHdrFlags, 4);
  std::memcpy(&seed, hdr + kHdrSeed, 8);
  ckpp_geometry g{nb, slots, flags, seed};
  if (magic != kMagic || abi != kAbiVersion || !geometry_ok(&g) || bytes < table_bytes(&g)) return CKPP_EINVAL;
  ckpp_table* t = new (std::nothrow) ckpp_table;
  if (!t) return CKPP_EINVAL;
  std::memset(t, 0, sizeof *t);
  t->geo = g;
  t->base = static_cast<uint8_t*>(dev_buf);
  t->bytes = table_bytes(&g);
  t->view.buckets = t->base + kHeaderBytes;
  t->view.err = reinterpret_cast<uint32_t*>(t->base + kHdrErr);
  t->view.nb = nb;
  t->view.seed = seed;
  t->view.timers = (flags & CKPP_TIMERS) ? 1u : 0u;
  t->have_epoch = t->view.timers ? 1 : 0;
  t->last_scan = now;
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
                               refresh_ttl, host_io, CKPP_LOOKUP_BLOOM, reinterpret_cast<cudaStream_t>(stream)));
}

int ckpp_bulk_lookup_variant(ckpp_table* t, const ckpp_key* keys, uint64_t n, uint64_t* out_vals, uint8_t* out_found,
                             uint32_t now, uint16_t refresh_ttl, int variant, ckpp_stream_t stream) {
  if (!t || check_keys(keys, n) || refresh_ttl >= kAliveWindow) return CKPP_EINVAL;
  if (variant < CKPP_LOOKUP_BLOOM || variant > CKPP_LOOKUP_PESSIMISTIC) return CKPP_EINVAL;
  if (n && (!out_vals || !out_found || !aligned(out_vals, 8))) return CKPP_EINVAL;
  if (int rc = time_check(t, now)) return rc;
  if (!n) return CKPP_OK;
  return cuda_rc(launch_lookup(t->view, reinterpret_cast<const uint8_t*>(keys), n, out_vals, out_found, now,
                               refresh_ttl, false, variant, reinterpret_cast<cudaStream_t>(stream)));
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
  return cuda_rc(launch_insert(one_table(t), reinterpret_cast<const uint8_t*>(keys), vals, n, now,
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
  return cuda_rc(launch_delete(one_table(t), reinterpret_cast<const uint8_t*>(keys), n, now, status, ws, s));
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

int ckpp_lookup_probe_counts(ckpp_table* t, const ckpp_key* keys, uint64_t n, uint32_t now, int variant,
                             uint64_t* d_counts, ckpp_stream_t stream) {
  if (!t || check_keys(keys, n) || !d_counts || !aligned(d_counts, 8)) return CKPP_EINVAL;
  if (variant < CKPP_LOOKUP_BLOOM || variant > CKPP_LOOKUP_PESSIMISTIC) return CKPP_EINVAL;
  if (int rc = time_check(t, now)) return rc;
  if (!n) return CKPP_OK;
  return cuda_rc(launch_probe_counts(t->view, reinterpret_cast<const uint8_t*>(keys), n, now, variant,
                                     reinterpret_cast<unsigned long long*>(d_counts),
                                     reinterpret_cast<cudaStream_t>(stream)));
}

// ------------------------------------------------------------ batched form

struct ckpp_batch {
  std::vector<ckpp_table*> tables;
  std::vector<TableView> host_views;  // kept alive for the copy to the device
  TableView* dev_views;
  unsigned long long* ctrl;           // the lookup kernel's chunk and finished-warp counters
  bool any_timers;                    // some table has timers
  int sms;
};

// Descriptor buffer: the table views, then a 256-byte control block.
size_t ckpp_batch_bytes(uint32_t n_tables) { return align_up((size_t)n_tables * sizeof(TableView), kAlign) + kAlign; }

int ckpp_batch_create(ckpp_batch** out, ckpp_table* const* tables, uint32_t n_tables, void* dev_buf, size_t bytes,
                      ckpp_stream_t stream) {
  if (!out || !tables || n_tables == 0 || !dev_buf || !aligned(dev_buf, kAlign) ||
      bytes < ckpp_batch_bytes(n_tables))
    return CKPP_EINVAL;
  for (uint32_t i = 0; i < n_tables; ++i)
    if (!tables[i]) return CKPP_EINVAL;
  ckpp_batch* b = new (std::nothrow) ckpp_batch;
  if (!b) return CKPP_EINVAL;
  b->tables.assign(tables, tables + n_tables);
  b->host_views.resize(n_tables);
  b->any_timers = false;
  for (uint32_t i = 0; i < n_tables; ++i) {
    b->host_views[i] = tables[i]->view;
    b->any_timers = b->any_timers || tables[i]->view.timers;
  }
  b->dev_views = static_cast<TableView*>(dev_buf);
  b->ctrl = reinterpret_cast<unsigned long long*>(static_cast<uint8_t*>(dev_buf) +
                                                  align_up((size_t)n_tables * sizeof(TableView), kAlign));
  int dev = 0;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      prepare_batched_lookup() != cudaSuccess ||
      cudaMemcpyAsync(b->dev_views, b->host_views.data(), n_tables * sizeof(TableView), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemsetAsync(b->ctrl, 0, kAlign, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    delete b;
    return CKPP_ECUDA;
  }
  *out = b;
  return CKPP_OK;
}

int ckpp_batch_destroy(ckpp_batch* b) {
  if (!b) return CKPP_EINVAL;
  delete b;
  return CKPP_OK;
}

int ckpp_batch_insert(ckpp_batch* b, const ckpp_key* keys, const uint32_t* table_ids, const uint64_t* vals, uint64_t n,
                      uint32_t now, uint16_t ttl, uint8_t* status, void* workspace, size_t workspace_bytes,
                      ckpp_stream_t stream) {
  if (!b || check_keys(keys, n) || ttl >= kAliveWindow) return CKPP_EINVAL;
  if (n && (!table_ids || !vals || !status || !aligned(vals, 8) || !aligned(table_ids, 4))) return CKPP_EINVAL;
  for (ckpp_table* t : b->tables)
    if (int rc = time_check(t, now)) return rc;
  if (!n) return CKPP_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Workspace ws;
  if (int rc = prepare_workspace(n, workspace, workspace_bytes, s, ws)) return rc;
  const TableSet ts{b->host_views[0], b->dev_views, table_ids, (uint32_t)b->tables.size()};
  return cuda_rc(launch_insert(ts, reinterpret_cast<const uint8_t*>(keys), vals, n, now, (now + ttl) & 0xFFFFu, status,
                               ws, s));
}

int ckpp_batch_delete(ckpp_batch* b, const ckpp_key* keys, const uint32_t* table_ids, uint64_t n, uint32_t now,
                      uint8_t* status, void* workspace, size_t workspace_bytes, ckpp_stream_t stream) {
  if (!b || check_keys(keys, n)) return CKPP_EINVAL;
  if (n && (!table_ids || !status || !aligned(table_ids, 4))) return CKPP_EINVAL;
  for (ckpp_table* t : b->tables)
    if (int rc = time_check(t, now)) return rc;
  if (!n) return CKPP_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Workspace ws;
  if (int rc = prepare_workspace(n, workspace, workspace_bytes, s, ws)) return rc;
  const TableSet ts{b->host_views[0], b->dev_views, table_ids, (uint32_t)b->tables.size()};
  return cuda_rc(launch_delete(ts, reinterpret_cast<const uint8_t*>(keys), n, now, status, ws, s));
}

int ckpp_batch_lookup(ckpp_batch* b, const ckpp_lookup_job* d_jobs, uint32_t max_jobs, const uint32_t* d_n_jobs,
                      uint32_t now, const ckpp_batch_tuning* tuning, ckpp_stream_t stream) {
  if (!b || max_jobs > kBatchMaxJobs || (max_jobs && !d_jobs)) return CKPP_EINVAL;
  ckpp_batch_tuning tn = tuning ? *tuning : ckpp_batch_tuning{1, 1, 2, 32};
  const uint32_t T = tn.threads_per_key, G = tn.group_depth;
  if (!(T == 1 || T == 2 || T == 4) || !(G == 1 || G == 2) || tn.blocks_per_sm < 1 || tn.blocks_per_sm > 4)
    return CKPP_EINVAL;
  const uint32_t P = 32 / T;  // lanes that own keys in a warp iteration
  if (tn.keys_per_warp != 0 && tn.keys_per_warp != P) return CKPP_EINVAL;
  for (ckpp_table* t : b->tables)
    if (int rc = time_check(t, now)) return rc;
  if (!max_jobs) return CKPP_OK;
  return cuda_rc(launch_batched_lookup(b->dev_views, (uint32_t)b->tables.size(), d_jobs, d_n_jobs, max_jobs, now,
                                       (int)T, (int)G, (int)P, b->any_timers, tn.blocks_per_sm * (uint32_t)b->sms,
                                       b->ctrl,
                                       reinterpret_cast<cudaStream_t>(stream)));
}

int ckpp_set_insert_launch(int mode) {
  const int prev = set_insert_launch(mode);
  return prev < 0 ? CKPP_EINVAL : prev;
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
