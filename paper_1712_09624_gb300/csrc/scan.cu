// Whole-table passes: header initialisation, the expiration scan of Sec. 4.2
// and table statistics (the quantities behind Fig. 2, Fig. 5 and Table 2).
// Both passes stream the bucket array once with one thread per bucket in a
// grid-stride loop sized to the SM count.
#include "mutate.cuh"

namespace ckpp {

namespace {

__global__ void init_header_kernel(uint8_t* base, uint64_t nb, uint32_t slots, uint32_t flags, uint64_t seed) {
  *reinterpret_cast<uint32_t*>(base + kHdrMagic) = kMagic;
  *reinterpret_cast<uint32_t*>(base + kHdrAbi) = kAbiVersion;
  *reinterpret_cast<uint64_t*>(base + kHdrBuckets) = nb;
  *reinterpret_cast<uint32_t*>(base + kHdrSlots) = slots;
  *reinterpret_cast<uint32_t*>(base + kHdrFlags) = flags;
  *reinterpret_cast<uint64_t*>(base + kHdrSeed) = seed;
  *reinterpret_cast<uint32_t*>(base + kHdrErr) = 0u;
}

// Sec. 4.2: delete every dead entry. A dead entry stored in its secondary
// bucket decrements its primary's moved counter, and the filter is reset when
// the counter reaches zero (Sec. 4.1); no filter bit is set during the scan.
__global__ void __launch_bounds__(256) expire_kernel(TableView t, uint32_t now, unsigned long long* n_expired) {
  uint32_t count = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  // Two buckets per thread per step, both buckets' words loaded before either
  // is examined: twice the reads in flight for this streaming pass.
  for (uint64_t bb = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; bb < t.nb; bb += 2 * stride) {
    uint32_t bk[2], ctrl[2];
    uint64_t e0[2] = {0, 0}, e1[2] = {0, 0};
    bool have[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const uint64_t b = bb + u * stride;
      have[u] = b < t.nb;
      bk[u] = have[u] ? (uint32_t)b : 0u;
      ctrl[u] = have[u] ? ld32_cg(ctrl_ptr(t, bk[u])) : 0u;
      if (have[u] && t.timers) ld128_cg(expiry_ptr(t, bk[u], 0), e0[u], e1[u]);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const uint32_t b = bk[u];
      const uint32_t busy = ctrl[u] & kBusyMask;
      const uint32_t dead = busy & ~alive_mask(e0[u], e1[u], now);
      if (!have[u] || !t.timers || !dead) continue;
      uint32_t displaced = (ctrl[u] >> kInsecShift) & dead;
      while (displaced) {
        const int s = __ffs(displaced) - 1;
        displaced &= displaced - 1;
        Key k;
        ld128_cg(key_ptr(t, b, s), k.k0, k.k1);
        const Addr a = address_of(k, t.nb, t.seed);
        if (atomicSub(moved_ptr(t, a.b1), 1u) == 1u)
          atomicExch(reinterpret_cast<unsigned long long*>(bloom_ptr(t, a.b1)), 0ull);
      }
      atomicAnd(ctrl_ptr(t, b), ~(dead | (dead << kInsecShift)));
      count += __popc(dead);
    }
  }
  count = __reduce_add_sync(0xFFFFFFFFu, count);
  if ((threadIdx.x & 31) == 0 && count && n_expired) atomicAdd(n_expired, (unsigned long long)count);
}

// out[0] occupied, [1] live, [2] in_secondary, [3] moved==0, [4] moved sum,
// [5] filter bits set, [6] sum of popcount^2, [7..22] moved histogram.
__global__ void __launch_bounds__(256) stats_kernel(TableView t, uint32_t now, unsigned long long* out) {
  __shared__ unsigned long long acc[7 + 16];
  for (int j = threadIdx.x; j < 7 + 16; j += blockDim.x) acc[j] = 0;
  __syncthreads();
  unsigned long long occ = 0, live = 0, insec = 0, mz = 0, msum = 0, bits = 0, popsq = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t bb = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; bb < t.nb; bb += stride) {
    const uint32_t b = (uint32_t)bb;
    uint64_t w[4];
    ld256_cg(bucket_ptr(t, b), w);
    const uint32_t ctrl = (uint32_t)w[3];
    const uint32_t moved = (uint32_t)(w[3] >> 32);
    const uint32_t busy = ctrl & kBusyMask;
    uint32_t alive = busy;
    if (t.timers) {
      uint64_t e0, e1;
      ld128_cg(expiry_ptr(t, b, 0), e0, e1);
      alive &= alive_mask(e0, e1, now);
    }
    const uint32_t pop = __popcll(w[2]);
    occ += __popc(busy);
    live += __popc(alive);
    insec += __popc((ctrl >> kInsecShift) & busy);
    mz += moved == 0;
    msum += moved;
    bits += pop;
    popsq += pop * pop;
    atomicAdd(&acc[7 + (moved < 15 ? moved : 15)], 1ull);
  }
  atomicAdd(&acc[0], occ);
  atomicAdd(&acc[1], live);
  atomicAdd(&acc[2], insec);
  atomicAdd(&acc[3], mz);
  atomicAdd(&acc[4], msum);
  atomicAdd(&acc[5], bits);
  atomicAdd(&acc[6], popsq);
  __syncthreads();
  for (int j = threadIdx.x; j < 7 + 16; j += blockDim.x)
    if (acc[j]) atomicAdd(out + j, acc[j]);
}

unsigned scan_blocks(uint64_t nb) {
  const uint64_t want = (nb + 255) / 256;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, 8ull * device_sm_count()));
}

}  // namespace

cudaError_t launch_init_header(uint8_t* base, uint64_t nb, uint32_t slots, uint32_t flags, uint64_t seed,
                               cudaStream_t s) {
  init_header_kernel<<<1, 1, 0, s>>>(base, nb, slots, flags, seed);
  return cudaGetLastError();
}

cudaError_t launch_expire(const TableView& t, uint32_t now, unsigned long long* n_expired, cudaStream_t s) {
  expire_kernel<<<scan_blocks(t.nb), 256, 0, s>>>(t, now, n_expired);
  return cudaGetLastError();
}

cudaError_t launch_stats(const TableView& t, uint32_t now, unsigned long long* out, cudaStream_t s) {
  stats_kernel<<<scan_blocks(t.nb), 256, 0, s>>>(t, now, out);
  return cudaGetLastError();
}

}  // namespace ckpp
