// Batched form: many independent tables, each with its own lookup batch, all
// served by one persistent kernel launch (the GPU counterpart of the paper's
// share-nothing setting of one private table per core, Sec. 2 and Sec. 5.3).
//
// Work list: a device array of jobs {keys, out_vals, out_found, n, table}; the
// job count may live in device memory, so one captured CUDA graph can be
// replayed while the caller rewrites jobs between replays. Every block scans
// the job sizes into a prefix array in shared memory; warps then take chunks
// of the flat key range [0, total) from a counter in the batch descriptor, in
// order (up to eight chunks per draw, so one counter can serve the whole
// grid), so that (as with a plain launch's short-lived blocks) the resident
// warps read keys and write results within one narrow window of the batch. A
// lane finds its key's job in the prefix array by galloping forward from the
// job of its previous key (keys are drawn in increasing order), and the warp
// runs the cooperative lookup of probe.cuh over keys of possibly different
// tables.
// The last warp to finish resets the counter for the next launch, so
// launches that use one batch descriptor must not overlap on the GPU.
// Tuning (picked by the autotuner):
//   threads per key  1, 2 or 4 lanes of the warp per key in an iteration:
//                    32 / threads_per_key lanes own keys, and all 32 lanes
//                    fetch their bucket lines (8 lanes of 16 bytes per
//                    128-byte line, four lines per warp instruction); more
//                    lanes per key means fewer keys and fewer registers'
//                    worth of probes per warp, for small jobs;
//   group depth      1 or 2 keys owned per owning lane, i.e. up to
//                    32 / threads_per_key x group_depth line requests a warp
//                    has in flight;
//   blocks per SM of the persistent grid.
// Every configuration runs the same method and returns the same results.
#include "probe.cuh"

namespace ckpp {

struct BatchJob {  // layout of ckpp_lookup_job
  const uint8_t* keys;
  uint64_t* out_vals;
  uint8_t* out_found;
  uint32_t n;
  uint32_t table;
};

namespace {

constexpr int kBatchThreads = 512;  // 16 warps share one copy of the job prefix array
constexpr unsigned long long kMaxChunksPerDraw = 8;

// Exclusive prefix sums of the first nj job sizes into prefix[0..nj].
__device__ void scan_jobs(const BatchJob* __restrict__ jobs, uint32_t nj, unsigned long long* prefix) {
  __shared__ unsigned long long warp_sums[kBatchThreads / 32];
  const uint32_t per = (nj + blockDim.x - 1) / blockDim.x;
  const uint32_t lo = min(nj, threadIdx.x * per), hi = min(nj, lo + per);
  unsigned long long local = 0;
  for (uint32_t j = lo; j < hi; ++j) local += jobs[j].n;
  // inclusive warp scan of the per-thread sums
  unsigned long long x = local;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, w, d);
      if (lane >= d) w += y;
    }
    if (lane < (int)(blockDim.x >> 5)) warp_sums[lane] = w;
  }
  __syncthreads();
  unsigned long long run = x - local + (warp ? warp_sums[warp - 1] : 0);
  for (uint32_t j = lo; j < hi; ++j) {
    prefix[j] = run;
    run += jobs[j].n;
  }
  if (threadIdx.x == blockDim.x - 1) prefix[nj] = run;
  __syncthreads();
}

// Index of the job holding flat key idx: the last j with prefix[j] <= idx,
// searched from hint, a job with prefix[hint] <= idx (the job of an earlier
// key of the same lane: a lane's keys only move forward through the batch).
// Usually idx is still in job hint; otherwise the search gallops forward to
// bracket idx, then bisects the bracket.
__device__ __forceinline__ uint32_t find_job(const unsigned long long* prefix, uint32_t nj, unsigned long long idx,
                                             uint32_t hint) {
  if (prefix[hint + 1] > idx) return hint;
  uint32_t lo = hint + 1, hi = nj, step = 1;  // prefix[lo] <= idx < prefix[hi]
  for (;;) {
    const uint32_t probe = lo + step;
    if (probe >= nj) break;
    if (prefix[probe] > idx) {
      hi = probe;
      break;
    }
    lo = probe;
    step <<= 1;
  }
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (prefix[mid] <= idx) lo = mid; else hi = mid;
  }
  return lo;
}

// One warp iteration: lane l < kpw owns flat keys wbase + g * kpw + l, g < G.
// hint: the job of the lane's last key so far (0 at the start).
template <int G, int kTM>
__device__ __forceinline__ void lookup_chunk(const TableView* __restrict__ tables, uint32_t n_tables,
                                             const BatchJob* __restrict__ jobs, const unsigned long long* prefix,
                                             uint32_t nj, unsigned long long total, unsigned long long wbase,
                                             uint32_t kpw, uint32_t now, uint64_t pol, uint32_t& hint,
                                             WarpStage<G>& S) {
  const uint32_t lane = threadIdx.x & 31;
  Probe p[G];
  bool act[G];
  uint32_t jobi[G];
  unsigned long long local[G];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const unsigned long long idx = wbase + (unsigned long long)g * kpw + lane;
    act[g] = lane < kpw && idx < total;
    jobi[g] = 0;
    local[g] = 0;
    if (act[g]) {
      jobi[g] = hint = find_job(prefix, nj, idx, hint);
      act[g] = jobs[jobi[g]].table < n_tables;  // jobs naming no table are skipped
    }
    TableView tv{};
    Key k{0, 0};
    if (act[g]) {
      local[g] = idx - prefix[jobi[g]];
      tv = tables[jobs[jobi[g]].table];
      k = ld_key_ro(jobs[jobi[g]].keys + 16 * local[g], pol);
    }
    probe_init(p[g], k, tv.buckets, tv.nb, tv.seed, tv.timers);
  }
  run_probes<kBloom, false, G, kTM>(p, act, now, S);
#pragma unroll
  for (int g = 0; g < G; ++g) {
    if (!act[g]) continue;
    const BatchJob& jb = jobs[jobi[g]];
    jb.out_vals[local[g]] = p[g].value;
    jb.out_found[local[g]] = p[g].found ? 1 : 0;
  }
}

// Dynamic shared memory: the job prefix array, then one line slab per warp
// (128-byte aligned).
__host__ __device__ __forceinline__ size_t stage_offset(uint32_t max_jobs) {
  return ((size_t)(max_jobs + 1) * sizeof(unsigned long long) + 127) & ~(size_t)127;
}

template <int G>
size_t batched_smem(uint32_t max_jobs) {
  return stage_offset(max_jobs) + (kBatchThreads / 32) * sizeof(WarpStage<G>);
}

// kTM: kNoTimers when no table of the batch has timers, else kTimersPerKey.
template <int G, int kTM>
__global__ void __launch_bounds__(kBatchThreads) batched_lookup_kernel(const TableView* __restrict__ tables,
                                                                       uint32_t n_tables,
                                                                       const BatchJob* __restrict__ jobs,
                                                                       const uint32_t* __restrict__ n_jobs_ptr,
                                                                       uint32_t max_jobs, uint32_t now, uint32_t kpw,
                                                                       unsigned long long* __restrict__ ctrl) {
  extern __shared__ __align__(128) unsigned long long prefix[];
  WarpStage<G>* stages =
      reinterpret_cast<WarpStage<G>*>(reinterpret_cast<uint8_t*>(prefix) + stage_offset(max_jobs));
  const uint32_t nj = n_jobs_ptr ? min(ld32_cg(n_jobs_ptr), max_jobs) : max_jobs;
  scan_jobs(jobs, nj, prefix);
  const unsigned long long total = prefix[nj];
  const uint64_t pol = policy_evict_first();
  const uint32_t lane = threadIdx.x & 31;
  const unsigned long long per_chunk = (unsigned long long)kpw * G;
  const unsigned long long chunks = (total + per_chunk - 1) / per_chunk;
  // Chunks per atomic draw: up to kMaxChunksPerDraw on large launches (one
  // counter word serves every warp of the grid), fewer on small ones, so that
  // every warp gets about four draws rather than a few warps all the work.
  const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
  unsigned long long per_draw = chunks / (4 * warps);
  per_draw = per_draw < 1 ? 1 : (per_draw > kMaxChunksPerDraw ? kMaxChunksPerDraw : per_draw);
  uint32_t hint = 0;  // chunks are drawn in increasing order, so a lane's keys only move forward
  for (;;) {
    unsigned long long c = 0;
    if (lane == 0) c = atomicAdd(ctrl, 1ull) * per_draw;
    c = __shfl_sync(kFull, c, 0);
    if (c >= chunks) break;
    const unsigned long long c_end = c + per_draw < chunks ? c + per_draw : chunks;
    for (; c < c_end; ++c)
      lookup_chunk<G, kTM>(tables, n_tables, jobs, prefix, nj, total, c * per_chunk, kpw, now, pol, hint,
                           stages[threadIdx.x >> 5]);
  }
  // Every warp has drawn past the last chunk before it counts itself out, so
  // the last one out can reset the counters for the next launch.
  if (lane == 0) {
    unsigned int* out = reinterpret_cast<unsigned int*>(ctrl + 1);
    if (atomicAdd(out, 1u) == (unsigned int)(warps - 1)) {
      atomicExch(ctrl, 0ull);
      atomicExch(out, 0u);
    }
  }
}

template <int G, int kTM>
cudaError_t set_smem_limit() {
  return cudaFuncSetAttribute(batched_lookup_kernel<G, kTM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)batched_smem<G>(kBatchMaxJobs));
}

template <int G, int kTM>
cudaError_t launch_g(const TableView* tables, uint32_t n_tables, const BatchJob* jobs, const uint32_t* n_jobs,
                     uint32_t max_jobs, uint32_t now, uint32_t kpw, uint32_t blocks, unsigned long long* ctrl,
                     cudaStream_t s) {
  batched_lookup_kernel<G, kTM><<<blocks, kBatchThreads, batched_smem<G>(max_jobs), s>>>(
      tables, n_tables, jobs, n_jobs, max_jobs, now, kpw, ctrl);
  return cudaGetLastError();
}

}  // namespace

cudaError_t prepare_batched_lookup() {
  cudaError_t e;
  if ((e = set_smem_limit<1, kNoTimers>()) != cudaSuccess) return e;
  if ((e = set_smem_limit<2, kNoTimers>()) != cudaSuccess) return e;
  if ((e = set_smem_limit<1, kTimersPerKey>()) != cudaSuccess) return e;
  return set_smem_limit<2, kTimersPerKey>();
}

cudaError_t launch_batched_lookup(const TableView* tables, uint32_t n_tables, const void* jobs, const uint32_t* n_jobs,
                                  uint32_t max_jobs, uint32_t now, int threads_per_key, int group_depth,
                                  int keys_per_warp, bool any_timers, uint32_t blocks, unsigned long long* ctrl,
                                  cudaStream_t s) {
  const BatchJob* j = static_cast<const BatchJob*>(jobs);
  if (!(threads_per_key == 1 || threads_per_key == 2 || threads_per_key == 4) ||
      keys_per_warp * threads_per_key != 32)
    return cudaErrorInvalidValue;
  const uint32_t kpw = (uint32_t)keys_per_warp;
  switch (group_depth * 2 + (any_timers ? 1 : 0)) {
    case 2: return launch_g<1, kNoTimers>(tables, n_tables, j, n_jobs, max_jobs, now, kpw, blocks, ctrl, s);
    case 3: return launch_g<1, kTimersPerKey>(tables, n_tables, j, n_jobs, max_jobs, now, kpw, blocks, ctrl, s);
    case 4: return launch_g<2, kNoTimers>(tables, n_tables, j, n_jobs, max_jobs, now, kpw, blocks, ctrl, s);
    case 5: return launch_g<2, kTimersPerKey>(tables, n_tables, j, n_jobs, max_jobs, now, kpw, blocks, ctrl, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ckpp
