// L2 read probe: the bandwidth at which the SMs can stream a buffer that sits
// in L2. A lookup batch on a table smaller than L2 (the 2^17-bucket table of
// the small configuration is 32 MiB) is served from L2, not HBM, so its
// roofline is this rate rather than the HBM copy bandwidth.
//
// Every thread reads 16-byte vectors with ld.global.cg (cached in L2 only, so
// L1 cannot serve repeats), four independent loads in flight per step, over a
// grid-stride walk of the buffer, `passes` times. The loaded words are folded
// into one value that is stored only if it equals a constant the data cannot
// produce, so that the loads cannot be dropped.
#include <cstdint>
#include <cuda_runtime.h>

#include "../../../include/ckpp_workload.h"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ uint4 ld16_cg(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}

__global__ void __launch_bounds__(kThreads) l2_read_kernel(const uint4* __restrict__ buf, uint64_t n_vec,
                                                           uint32_t passes, unsigned long long* sink) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  for (uint32_t p = 0; p < passes; ++p) {
    uint64_t i = tid;
    for (; i + 3 * stride < n_vec; i += 4 * stride) {
      const uint4 a = ld16_cg(buf + i), b = ld16_cg(buf + i + stride), c = ld16_cg(buf + i + 2 * stride),
                  d = ld16_cg(buf + i + 3 * stride);
      acc ^= a.x ^ a.w ^ b.y ^ b.z ^ c.x ^ c.w ^ d.y ^ d.z;
    }
    for (; i < n_vec; i += stride) {
      const uint4 a = ld16_cg(buf + i);
      acc ^= a.x ^ a.y ^ a.z ^ a.w;
    }
  }
  if (acc == 0x9E3779B9u && sink) atomicAdd(sink, 1ull);
}

}  // namespace

extern "C" int ckpp_wl_l2_read(const uint8_t* buf, uint64_t bytes, uint32_t passes, uint64_t* sink,
                               ckpp_wl_stream_t stream) {
  if (!buf || bytes == 0 || bytes % 16 != 0 || (reinterpret_cast<uintptr_t>(buf) % 16) != 0 || passes == 0)
    return -1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess) {
    cudaGetLastError();
    return -2;
  }
  l2_read_kernel<<<(unsigned)sms * 8, kThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const uint4*>(buf), bytes / 16, passes, reinterpret_cast<unsigned long long*>(sink));
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
