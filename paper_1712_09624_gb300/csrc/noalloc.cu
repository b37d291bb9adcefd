// ckpp_bulk_insert_noalloc: bulk insert whose scratch lives in a fixed device
// array compiled into this library, for callers that cannot allocate.
//
// ckpp_bulk_insert needs a workspace buffer from the caller. Some callers have
// no way to get one at the time they insert: a data-plane thread that owns a
// fixed memory budget handed out at start-up and must never call cudaMalloc or
// cudaFree (cudaFree can stall the whole device), or a plugin running inside a
// host framework that owns all device memory and exposes no allocator. This
// entry point takes the same inputs and outputs and uses, instead of a
// workspace, the file-scope array below: kNoallocBytes of device memory that
// every GPU which loads libckpp.so keeps until the process exits.
//
// The paper has no counterpart to this entry point; it only changes where the
// batch's scratch memory comes from.
#include <mutex>

#include "api_internal.h"

using namespace ckpp;
using namespace ckpp::api;

namespace {

constexpr uint64_t kNoallocMaxKeys = CKPP_NOALLOC_MAX_KEYS;
constexpr size_t kNoallocBytes = ws_layout(kNoallocMaxKeys).total;

// The scratch array. In host code its name is only a host-side stand-in, not
// a device address: the address kernels must use comes from
// cudaGetSymbolAddress, taken once per device below.
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Address of the scratch array on the current device (set-up on first use).
// The address is cached for the life of the process: after cudaDeviceReset the
// module is loaded again and the cached address is no longer valid, so a
// process that resets a device must reload libckpp.so before calling again.
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CKPP_ECUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();  // clear it, so that a later call's launch check does not report it
      return CKPP_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return CKPP_OK;
}

}  // namespace

extern "C" int ckpp_bulk_insert_noalloc(ckpp_table* t, const ckpp_key* keys, const uint64_t* vals, uint64_t n,
                                        uint32_t now, uint16_t ttl, uint8_t* status, ckpp_stream_t stream) {
  if (!t || check_keys(keys, n) || ttl >= kAliveWindow || n > kNoallocMaxKeys) return CKPP_EINVAL;
  if (n && (!vals || !status || !aligned(vals, 8))) return CKPP_EINVAL;
  if (int rc = time_check(t, now)) return rc;
  if (!n) return CKPP_OK;
  void* scratch = nullptr;
  if (int rc = scratch_address(&scratch)) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Workspace ws;
  // prepare_workspace clears the counters and the duplicate-key set, the parts
  // that must start at zero (the array keeps the previous call's contents).
  if (int rc = prepare_workspace(n, scratch, kNoallocBytes, s, ws)) return rc;
  return cuda_rc(launch_insert(one_table(t), reinterpret_cast<const uint8_t*>(keys), vals, n, now,
                               (now + ttl) & 0xFFFFu, status, ws, s));
}
