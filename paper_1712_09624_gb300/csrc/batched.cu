// Batched form: many independent tables, each with its own lookup batch, all
// served by one persistent kernel launch (the GPU counterpart of the paper's
// share-nothing setting of one private table per core, Sec. 2 and Sec. 5.3).
//
// Work list: a device array of jobs {keys, out_vals, out_found, n, table}; the
// job count may live in device memory, so one captured CUDA graph can be
// replayed while the caller rewrites jobs between replays. Every block scans
// the job sizes into a prefix array in shared memory and then walks the flat
// key range [0, total) in warp-sized chunks with a grid-stride loop; a key finds
// its job by binary search in the prefix array.
//
// Tuning (picked by the autotuner):
//   T  threads per key (1, 2, 4, 8): the T lanes of a group read the same bucket
//      sector and split its 8 slots between them (slot s goes to lane s mod T),
//      then combine with a warp ballot;
//   G  group depth (1, 2, 4; T = 1 only): each thread issues the primary-bucket
//      and first-record reads of G keys before consuming any of them;
//   blocks per SM of the persistent grid.
// Every configuration runs the method of probe.cuh and returns the same results.
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

constexpr int kBatchThreads = 256;

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

// Index of the job holding flat key idx: the last j with prefix[j] <= idx.
__device__ __forceinline__ uint32_t find_job(const unsigned long long* prefix, uint32_t nj, unsigned long long idx) {
  uint32_t lo = 0, hi = nj;  // prefix[lo] <= idx < prefix[hi]
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (prefix[mid] <= idx) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ TableView load_view(const TableView* tables, uint32_t i) { return tables[i]; }

// One key per thread (T = 1), G keys in flight per thread.
template <int G>
__device__ void lookup_g(const TableView* __restrict__ tables, uint32_t n_tables, const BatchJob* __restrict__ jobs,
                         const unsigned long long* prefix, uint32_t nj, unsigned long long total,
                         unsigned long long wbase, uint32_t now, uint64_t keep, uint64_t stream) {
  const uint32_t lane = threadIdx.x & 31;
  bool act[G];
  uint32_t job[G];
  unsigned long long local[G];
  Key k[G];
  TableView tv[G];
  Addr a[G];
  uint64_t h[G][4];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const unsigned long long idx = wbase + (unsigned long long)g * 32 + lane;
    act[g] = idx < total;
    job[g] = act[g] ? find_job(prefix, nj, idx) : 0;
    local[g] = act[g] ? idx - prefix[job[g]] : 0;
    act[g] = act[g] && jobs[job[g]].table < n_tables;  // jobs naming no table are skipped
  }
#pragma unroll
  for (int g = 0; g < G; ++g) {
    if (!act[g]) continue;
    tv[g] = load_view(tables, jobs[job[g]].table);
    k[g] = ld_key_ro(jobs[job[g]].keys + 16 * local[g], stream);
  }
#pragma unroll
  for (int g = 0; g < G; ++g) {
    if (!act[g]) continue;
    a[g] = address_of(k[g], tv[g].nb, tv[g].seed);
    ld256_ro(bucket_ptr(tv[g], a[g].b1), keep, h[g]);
  }
  // first candidate record of every key, all in flight together
  uint64_t rec[G][4];
  uint32_t cand[G];
  int first[G];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    first[g] = -1;
    if (!act[g]) continue;
    cand[g] = candidates(h[g], a[g].tag);
    if (cand[g]) {
      first[g] = __ffs(cand[g]) - 1;
      cand[g] &= cand[g] - 1;
      ld256_ro(record_ptr(tv[g], a[g].b1, first[g]), stream, rec[g]);
    }
  }
#pragma unroll
  for (int g = 0; g < G; ++g) {
    if (!act[g]) continue;
    const BatchJob& jb = jobs[job[g]];
    uint32_t b = a[g].b1, expiry = 0, nrec = 0;
    int s = (first[g] >= 0 && same_key(rec[g], k[g])) ? first[g] : -1;
    if (s < 0 && cand[g]) {
      s = tv[g].timers ? confirm<true, false>(tv[g], b, cand[g], k[g], stream, rec[g], expiry, nrec)
                       : confirm<false, false>(tv[g], b, cand[g], k[g], stream, rec[g], expiry, nrec);
    }
    if (s < 0 && (h[g][2] & a[g].bits) == a[g].bits) {
      uint64_t h2[4];
      b = a[g].b2;
      ld256_ro(bucket_ptr(tv[g], b), keep, h2);
      s = tv[g].timers ? confirm<true, false>(tv[g], b, candidates(h2, a[g].tag), k[g], stream, rec[g], expiry, nrec)
                       : confirm<false, false>(tv[g], b, candidates(h2, a[g].tag), k[g], stream, rec[g], expiry, nrec);
    }
    bool found = s >= 0;
    if (found && tv[g].timers) found = alive16((uint32_t)(rec[g][3] & 0xFFFFu), now);
    jb.out_vals[local[g]] = found ? rec[g][2] : 0ull;
    jb.out_found[local[g]] = found ? 1 : 0;
  }
}

// T lanes per key: lane r of a group handles the slots s with s % T == r.
template <int T>
__device__ void lookup_t(const TableView* __restrict__ tables, uint32_t n_tables, const BatchJob* __restrict__ jobs,
                         const unsigned long long* prefix, uint32_t nj, unsigned long long total,
                         unsigned long long wbase, uint32_t now, uint64_t keep, uint64_t stream) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t r = lane % T, gbase = lane - r;
  const uint32_t gmask = ((1u << T) - 1u) << gbase;
  uint32_t own = 0;
#pragma unroll
  for (int s = 0; s < (int)kSlots; ++s) own |= ((uint32_t)(s % T) == r ? 1u : 0u) << s;
  const unsigned long long idx = wbase + lane / T;
  bool act = idx < total;
  uint32_t jobi = 0;
  unsigned long long local = 0;
  if (act) {
    jobi = find_job(prefix, nj, idx);
    act = jobs[jobi].table < n_tables;  // jobs naming no table are skipped
  }
  TableView tv{};
  Key k{0, 0};
  Addr a{};
  uint64_t h[4] = {0, 0, 0, 0}, rec[4] = {0, 0, 0, 0};
  if (act) {
    local = idx - prefix[jobi];
    tv = load_view(tables, jobs[jobi].table);
    k = ld_key_ro(jobs[jobi].keys + 16 * local, stream);
    a = address_of(k, tv.nb, tv.seed);
    ld256_ro(bucket_ptr(tv, a.b1), keep, h);
  }
  uint32_t b = a.b1, expiry = 0, nrec = 0;
  int s = -1;
  if (act) {
    s = tv.timers ? confirm<true, false>(tv, b, candidates(h, a.tag) & own, k, stream, rec, expiry, nrec)
                  : confirm<false, false>(tv, b, candidates(h, a.tag) & own, k, stream, rec, expiry, nrec);
  }
  uint32_t hits = __ballot_sync(0xFFFFFFFFu, s >= 0) & gmask;
  const bool need2 = act && !hits && (h[2] & a.bits) == a.bits;
  if (need2) {
    uint64_t h2[4];
    b = a.b2;
    ld256_ro(bucket_ptr(tv, b), keep, h2);
    s = tv.timers ? confirm<true, false>(tv, b, candidates(h2, a.tag) & own, k, stream, rec, expiry, nrec)
                  : confirm<false, false>(tv, b, candidates(h2, a.tag) & own, k, stream, rec, expiry, nrec);
  }
  hits |= __ballot_sync(0xFFFFFFFFu, need2 && s >= 0) & gmask;
  bool found = s >= 0;
  if (found && tv.timers) found = alive16(expiry, now);
  const uint32_t src = hits ? (uint32_t)(__ffs(hits) - 1) : lane;
  const uint64_t value = __shfl_sync(0xFFFFFFFFu, found ? rec[2] : 0ull, src);
  const int fsrc = __shfl_sync(0xFFFFFFFFu, found ? 1 : 0, src);
  if (act && r == 0) {
    const BatchJob& jb = jobs[jobi];
    jb.out_vals[local] = hits ? value : 0ull;
    jb.out_found[local] = hits ? (uint8_t)fsrc : 0;
  }
}

template <int T, int G>
__global__ void __launch_bounds__(kBatchThreads) batched_lookup_kernel(const TableView* __restrict__ tables,
                                                                       uint32_t n_tables,
                                                                       const BatchJob* __restrict__ jobs,
                                                                       const uint32_t* __restrict__ n_jobs_ptr,
                                                                       uint32_t max_jobs, uint32_t now) {
  extern __shared__ unsigned long long prefix[];
  const uint32_t nj = n_jobs_ptr ? min(ld32_cg(n_jobs_ptr), max_jobs) : max_jobs;
  scan_jobs(jobs, nj, prefix);
  const unsigned long long total = prefix[nj];
  const uint64_t keep = policy_evict_last();
  const uint64_t stream = policy_evict_first();
  const unsigned long long per_warp = (unsigned long long)(32 / T) * G;
  const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
  for (unsigned long long w = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
       w * per_warp < total; w += warps) {
    if (T == 1) {
      lookup_g<G>(tables, n_tables, jobs, prefix, nj, total, w * per_warp, now, keep, stream);
    } else {
      lookup_t<T>(tables, n_tables, jobs, prefix, nj, total, w * per_warp, now, keep, stream);
    }
  }
}

template <int T, int G>
cudaError_t set_smem_limit() {
  return cudaFuncSetAttribute(batched_lookup_kernel<T, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)((kBatchMaxJobs + 1) * sizeof(unsigned long long)));
}

template <int T, int G>
cudaError_t launch_tg(const TableView* tables, uint32_t n_tables, const BatchJob* jobs, const uint32_t* n_jobs,
                      uint32_t max_jobs, uint32_t now, uint32_t blocks, cudaStream_t s) {
  const size_t smem = (size_t)(max_jobs + 1) * sizeof(unsigned long long);
  batched_lookup_kernel<T, G><<<blocks, kBatchThreads, smem, s>>>(tables, n_tables, jobs, n_jobs, max_jobs, now);
  return cudaGetLastError();
}

}  // namespace

cudaError_t prepare_batched_lookup() {
  cudaError_t e;
  if ((e = set_smem_limit<1, 1>()) != cudaSuccess) return e;
  if ((e = set_smem_limit<1, 2>()) != cudaSuccess) return e;
  if ((e = set_smem_limit<1, 4>()) != cudaSuccess) return e;
  if ((e = set_smem_limit<2, 1>()) != cudaSuccess) return e;
  if ((e = set_smem_limit<4, 1>()) != cudaSuccess) return e;
  return set_smem_limit<8, 1>();
}

cudaError_t launch_batched_lookup(const TableView* tables, uint32_t n_tables, const void* jobs, const uint32_t* n_jobs,
                                  uint32_t max_jobs, uint32_t now, int threads_per_key, int group_depth,
                                  uint32_t blocks, cudaStream_t s) {
  const BatchJob* j = static_cast<const BatchJob*>(jobs);
  switch (threads_per_key * 16 + group_depth) {
    case 1 * 16 + 1: return launch_tg<1, 1>(tables, n_tables, j, n_jobs, max_jobs, now, blocks, s);
    case 1 * 16 + 2: return launch_tg<1, 2>(tables, n_tables, j, n_jobs, max_jobs, now, blocks, s);
    case 1 * 16 + 4: return launch_tg<1, 4>(tables, n_tables, j, n_jobs, max_jobs, now, blocks, s);
    case 2 * 16 + 1: return launch_tg<2, 1>(tables, n_tables, j, n_jobs, max_jobs, now, blocks, s);
    case 4 * 16 + 1: return launch_tg<4, 1>(tables, n_tables, j, n_jobs, max_jobs, now, blocks, s);
    case 8 * 16 + 1: return launch_tg<8, 1>(tables, n_tables, j, n_jobs, max_jobs, now, blocks, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ckpp
