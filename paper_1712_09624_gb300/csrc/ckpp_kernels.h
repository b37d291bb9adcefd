// Internal launchers of the GB300 Cuckoo++ kernels (host side, C++).
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "ckpp_device.cuh"

namespace ckpp {

// Streaming multiprocessors of the current device, queried once per device
// and cached (grid sizes of the grid-stride and persistent kernels are
// multiples of it). A failed query is not cached and returns 1, which keeps a
// grid valid; the launch that follows reports the device's error.
inline int device_sm_count() {
  constexpr int kMaxDevices = 64;
  static std::atomic<int> cache[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return 1;
  }
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
    cudaGetLastError();
    return 1;
  }
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

// Device scratch for one insert or delete batch (carved out of the caller's
// workspace buffer, see workspace_layout in api.cu).
struct Workspace {
  uint32_t* counters;   // [0] pending count, [1] fixup count, [2] fixup overflow flag; list counts of the
                        // displacement passes: [3] after move1 (in `retry`), [5] after the grid search
                        // (in `pending`), [6] after the second search (in `retry`)
  uint32_t* set;        // [2m] open-addressing set of batch keys; position p holds two words side by
                        // side (one line for both): the lowest batch index of the key (kEmpty when
                        // free) and the highest
  uint32_t* slot_of;    // [n] set position of each batch key
  uint8_t* dup;         // [n] 1 when the key's group has other members (cleared to 0 with the set)
  uint32_t* pending;    // [n] leaders left for the displacement pass
  uint32_t* retry;      // [n] leaders a displacement pass passes on to the next
  unsigned long long* claim;  // [n] per key: (bucket << 32) | the ctrl bits its publication flips, or 0
                              // (the slot phase 1 claimed for it; written by phase 1 for every key)
  unsigned long long* fixup;  // [fix_cap] (table << 32 | bucket) whose moved counter fell to 0 off-lock
  uint32_t m_mask;      // m - 1 (m a power of two >= 4n)
  uint32_t fix_cap;

  __device__ __forceinline__ uint32_t* first_at(uint32_t p) const { return set + 2 * (uint64_t)p; }
  __device__ __forceinline__ uint32_t* last_at(uint32_t p) const { return set + 2 * (uint64_t)p + 1; }
  // both words of position p as one 64-bit word: first in the low half, last in the high half
  __device__ __forceinline__ unsigned long long* pair_at(uint32_t p) const {
    return reinterpret_cast<unsigned long long*>(set + 2 * (uint64_t)p);
  }
};

// The table(s) a mutation batch works on: one table, or many (key i goes to
// views[tab[i]]; keys naming no table are reported CKPP_ST_NO_TABLE).
struct TableSet {
  TableView single;
  const TableView* views;  // nullptr: every key goes to `single`
  const uint32_t* tab;     // per-key table index when views != nullptr
  uint32_t n_tables;

  __device__ __forceinline__ bool valid(uint64_t i) const { return !views || tab[i] < n_tables; }
  __device__ __forceinline__ uint32_t id(uint64_t i) const { return views ? tab[i] : 0u; }
  __device__ __forceinline__ TableView of(uint64_t i) const { return views ? views[tab[i]] : single; }
  __device__ __forceinline__ TableView table(uint32_t id) const { return views ? views[id] : single; }
};

cudaError_t launch_init_header(uint8_t* base, uint64_t nb, uint32_t slots, uint32_t flags, uint64_t seed,
                               cudaStream_t s);

// host_io: keys and outputs are pinned host memory (read and written in place
// over NVLink-C2C). variant: 0 Cuckoo++ (filter-pruned), 1 optimistic,
// 2 pessimistic (probe.cuh).
cudaError_t launch_lookup(const TableView& t, const uint8_t* keys, uint64_t n, uint64_t* out_vals,
                          uint8_t* out_found, uint32_t now, uint32_t refresh_ttl, bool host_io, int variant,
                          cudaStream_t s);

cudaError_t launch_probe_counts(const TableView& t, const uint8_t* keys, uint64_t n, uint32_t now, int variant,
                                unsigned long long* counts, cudaStream_t s);

// Batched form (batched.cu): tables [n_tables] in device memory, jobs a device
// array of ckpp_lookup_job, n_jobs NULL or a device count (clamped to max_jobs),
// ctrl the descriptor's two zeroed counter words (chunk counter, warps done).
cudaError_t prepare_batched_lookup();
cudaError_t launch_batched_lookup(const TableView* tables, uint32_t n_tables, const void* jobs, const uint32_t* n_jobs,
                                  uint32_t max_jobs, uint32_t now, int threads_per_key, int group_depth,
                                  int keys_per_warp, bool any_timers, uint32_t blocks, unsigned long long* ctrl,
                                  cudaStream_t s);

// Resets a carved workspace for a new batch: counter_words counters to 0, the
// dedup set's first-index words to empty and last-index words to 0 (one launch).
cudaError_t launch_workspace_clear(const Workspace& ws, uint32_t counter_words, uint64_t n, cudaStream_t s);

cudaError_t launch_dedup(const TableSet& ts, const uint8_t* keys, uint64_t n, const Workspace& ws,
                         cudaStream_t s);

// An insert call runs as a chain of kernels (the default) or as one
// cooperative launch (insert.cu), whichever mode the caller picks.
constexpr int kInsertLaunchChain = 0, kInsertLaunchSingle = 1;
int set_insert_launch(int mode);  // returns the previous mode, or -1 for an unknown mode

cudaError_t launch_insert(const TableSet& ts, const uint8_t* keys, const uint64_t* vals, uint64_t n,
                          uint32_t now, uint32_t expiry, uint8_t* status, const Workspace& ws, cudaStream_t s);

cudaError_t launch_delete(const TableSet& ts, const uint8_t* keys, uint64_t n, uint32_t now, uint8_t* status,
                          const Workspace& ws, cudaStream_t s);

cudaError_t launch_expire(const TableView& t, uint32_t now, unsigned long long* n_expired, cudaStream_t s);

// out: 7 sums + 16 histogram bins (uint64), zeroed by the caller.
cudaError_t launch_stats(const TableView& t, uint32_t now, unsigned long long* out, cudaStream_t s);

}  // namespace ckpp
