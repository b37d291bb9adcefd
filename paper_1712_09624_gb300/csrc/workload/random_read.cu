// Random-read probe: the rate at which this GPU serves independent random
// reads of 32 or 64 bytes from a large buffer. It measures the ceiling that
// bounds a hash-table lookup (a few random sectors per key), next to the
// sequential copy bandwidth used as the roofline peak.
#include <cstdint>
#include <cuda_runtime.h>

#include "../../../include/ckpp_workload.h"

namespace {

__device__ __forceinline__ uint64_t scramble(uint64_t z) {  // a cheap bijective 64-bit mixer
  z ^= z >> 33;
  z *= 0xFF51AFD7ED558CCDull;
  z ^= z >> 33;
  z *= 0xC4CEB9FE1A85EC53ull;
  z ^= z >> 33;
  return z;
}

template <int kUnit>
__global__ void random_read_kernel(const uint8_t* __restrict__ buf, uint64_t units_mask, uint64_t n, uint64_t seed,
                                   unsigned long long* sink) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint8_t* p = buf + (scramble(seed + i) & units_mask) * kUnit;
  uint64_t a, b, c, d, acc;
  asm volatile("ld.global.nc.v4.u64 {%0,%1,%2,%3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
  acc = a ^ b ^ c ^ d;
  if (kUnit == 64) {
    asm volatile("ld.global.nc.v4.u64 {%0,%1,%2,%3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p + 32));
    acc ^= a ^ b ^ c ^ d;
  }
  if (acc == 0x9E3779B97F4A7C15ull) atomicAdd(sink, 1ull);  // keeps the loads live
}

// Line-read probe: what one random access costs by request shape. Every mode
// makes n "accesses" (a group of lanes or one lane); see ckpp_workload.h.
__device__ __forceinline__ void ld32(const uint8_t* p, uint64_t (&w)[4]) {
  asm volatile("ld.global.nc.L1::no_allocate.v4.u64 {%0,%1,%2,%3}, [%4];"
               : "=l"(w[0]), "=l"(w[1]), "=l"(w[2]), "=l"(w[3]) : "l"(p));
}
__device__ __forceinline__ void ld32_p128(const uint8_t* p, uint64_t (&w)[4]) {
  asm volatile("ld.global.nc.L1::no_allocate.L2::128B.v4.u64 {%0,%1,%2,%3}, [%4];"
               : "=l"(w[0]), "=l"(w[1]), "=l"(w[2]), "=l"(w[3]) : "l"(p));
}

__host__ __device__ constexpr int lanes_of(int mode) { return mode == 2 ? 4 : mode == 3 ? 8 : 1; }

template <int kMode>
__global__ void __launch_bounds__(256) line_read_kernel(const uint8_t* __restrict__ buf, uint64_t bytes, uint64_t n,
                                                        uint64_t seed, unsigned long long* sink) {
  constexpr int L = lanes_of(kMode);
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t g = t / L;
  const uint32_t lane = (uint32_t)(t % L);
  if (g >= n) return;
  uint64_t w[4], v[4], acc;
  if (kMode == 0) {
    ld32(buf + (scramble(seed + g) & (bytes / 32 - 1)) * 32, w);
    acc = w[0] ^ w[3];
  } else if (kMode == 1) {
    const uint8_t* p = buf + (scramble(seed + g) & (bytes / 64 - 1)) * 64;
    ld32(p, w);
    ld32(p + 32, v);
    acc = w[0] ^ v[3];
  } else if (kMode == 2 || kMode == 3) {
    const uint64_t unit = 32ull * L;
    ld32(buf + (scramble(seed + g) & (bytes / unit - 1)) * unit + 32ull * lane, w);
    acc = w[0] ^ w[3];
  } else {  // 4, 5: a 32-byte read, then one that depends on it, in the same 128-byte line
    const uint64_t off = (scramble(seed + g) & (bytes / 128 - 1)) * 128;
    if (kMode == 4) ld32(buf + off, w); else ld32_p128(buf + off, w);
    ld32(buf + off + 32 + (w[0] & 32), v);  // the buffer is zero: off + 32
    acc = w[1] ^ v[2];
  }
  if (acc == 0x9E3779B97F4A7C15ull) atomicAdd(sink, 1ull);
}

// Mode 6: each warp stages 32 random lines in shared memory with cp.async, 8
// lanes x 16 bytes per line (four lines per instruction), then reads them.
__global__ void __launch_bounds__(256) line_stage_kernel(const uint8_t* __restrict__ buf, uint64_t bytes, uint64_t n,
                                                         uint64_t seed, unsigned long long* sink) {
  __shared__ __align__(128) uint8_t lines[8][32 * 128];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t g0 = (blockIdx.x * 8ull + warp) * 32;  // first line of this warp
  if (g0 >= n) return;
  const uint64_t mask = bytes / 128 - 1;
  for (uint32_t i = 0; i < 8; ++i) {
    const uint32_t j = 4 * i + (lane >> 3), c = lane & 7;
    if (g0 + j < n) {
      const uint8_t* src = buf + (scramble(seed + g0 + j) & mask) * 128 + 16 * c;
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&lines[warp][j * 128 + 16 * c]);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncwarp();
  const uint64_t acc = *reinterpret_cast<const uint64_t*>(&lines[warp][lane * 128 + 8 * (lane & 15)]);
  if (acc == 0x9E3779B97F4A7C15ull) atomicAdd(sink, 1ull);
}

}  // namespace

extern "C" int ckpp_wl_line_read(const uint8_t* buf, uint64_t bytes, int mode, uint64_t n, uint64_t seed,
                                 uint64_t* sink, ckpp_wl_stream_t stream) {
  if (!buf || !sink || mode < 0 || mode > 6 || bytes < 256 || (bytes & (bytes - 1)) ||
      reinterpret_cast<uintptr_t>(buf) % 256)
    return -1;
  if (n == 0) return 0;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned long long* k = reinterpret_cast<unsigned long long*>(sink);
  const uint64_t threads = mode == 6 ? (n + 31) / 32 * 32 : n * (uint64_t)(mode == 2 ? 4 : mode == 3 ? 8 : 1);
  const unsigned blocks = (unsigned)((threads + 255) / 256);
  switch (mode) {
    case 0: line_read_kernel<0><<<blocks, 256, 0, s>>>(buf, bytes, n, seed, k); break;
    case 1: line_read_kernel<1><<<blocks, 256, 0, s>>>(buf, bytes, n, seed, k); break;
    case 2: line_read_kernel<2><<<blocks, 256, 0, s>>>(buf, bytes, n, seed, k); break;
    case 3: line_read_kernel<3><<<blocks, 256, 0, s>>>(buf, bytes, n, seed, k); break;
    case 4: line_read_kernel<4><<<blocks, 256, 0, s>>>(buf, bytes, n, seed, k); break;
    case 5: line_read_kernel<5><<<blocks, 256, 0, s>>>(buf, bytes, n, seed, k); break;
    default: line_stage_kernel<<<blocks, 256, 0, s>>>(buf, bytes, n, seed, k); break;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

extern "C" int ckpp_wl_random_read(const uint8_t* buf, uint64_t bytes, uint32_t unit, uint64_t n, uint64_t seed,
                                   uint64_t* sink, ckpp_wl_stream_t stream) {
  if (!buf || !sink || (unit != 32 && unit != 64) || bytes < unit || (bytes & (bytes - 1)) ||
      reinterpret_cast<uintptr_t>(buf) % 64)
    return -1;
  if (n == 0) return 0;
  const uint64_t mask = bytes / unit - 1;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (unit == 32)
    random_read_kernel<32><<<blocks, 256, 0, s>>>(buf, mask, n, seed, reinterpret_cast<unsigned long long*>(sink));
  else
    random_read_kernel<64><<<blocks, 256, 0, s>>>(buf, mask, n, seed, reinterpret_cast<unsigned long long*>(sink));
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
