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

}  // namespace

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
