// Host-link probe: the host I/O of a lookup whose keys and results live in
// pinned host memory, without the table. Each lane reads one 16-byte key over
// NVLink-C2C and each warp writes its 32 results back as 16-byte vectors (the
// access pattern of ckpp_bulk_lookup on host buffers); the value and flag are
// derived from the key alone. Its rate is the ceiling of such a lookup.
#include <cstdint>
#include <cuda_runtime.h>

#include "../../../include/ckpp_workload.h"

namespace {

constexpr int kThreads = 128;

__global__ void __launch_bounds__(kThreads) host_io_kernel(const uint8_t* __restrict__ keys, uint64_t n,
                                                           uint64_t* __restrict__ out_vals,
                                                           uint8_t* __restrict__ out_found, bool vec) {
  __shared__ __align__(16) uint64_t vals[kThreads];
  __shared__ __align__(16) uint8_t flags[kThreads];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t c = (uint64_t)blockIdx.x * (kThreads / 32) + warp;  // the warp's 32-key chunk
  const uint64_t i = c * 32 + lane;
  uint64_t v = 0;
  uint8_t f = 0;
  if (i < n) {
    const ulonglong2 k = *reinterpret_cast<const ulonglong2*>(keys + 16 * i);
    v = k.x ^ (k.y << 1);
    f = (uint8_t)(k.y & 1u);
  }
  if (vec && c * 32 + 32 <= n) {
    vals[threadIdx.x] = v;
    flags[threadIdx.x] = f;
    __syncwarp();
    if (lane < 16) {
      reinterpret_cast<ulonglong2*>(out_vals + c * 32)[lane] = reinterpret_cast<const ulonglong2*>(vals + warp * 32)[lane];
    } else if (lane < 18) {
      reinterpret_cast<uint4*>(out_found + c * 32)[lane - 16] = reinterpret_cast<const uint4*>(flags + warp * 32)[lane - 16];
    }
  } else if (i < n) {
    out_vals[i] = v;
    out_found[i] = f;
  }
}

}  // namespace

extern "C" int ckpp_wl_host_io(const uint8_t* keys, uint64_t n, uint64_t* out_vals, uint8_t* out_found,
                               ckpp_wl_stream_t stream) {
  if (n == 0) return 0;
  if (!keys || !out_vals || !out_found || reinterpret_cast<uintptr_t>(keys) % 16 ||
      reinterpret_cast<uintptr_t>(out_vals) % 8)
    return -1;
  const bool vec = reinterpret_cast<uintptr_t>(out_vals) % 16 == 0 && reinterpret_cast<uintptr_t>(out_found) % 16 == 0;
  const uint64_t blocks = ((n + 31) / 32 + kThreads / 32 - 1) / (kThreads / 32);
  host_io_kernel<<<(unsigned)blocks, kThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(keys, n, out_vals,
                                                                                            out_found, vec);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
