// Device-side layout, hashing and memory helpers of the GB300 Cuckoo++ table.
//
// HBM layout of one table (caller-owned buffer, 256-byte aligned):
//   [0, 256)             header: magic, geometry copy, latched device error word
//   buckets              n_buckets buckets of 256 bytes: two 128-byte lines
//
// The paper keeps every field a bucket lookup reads in one cache line and the
// keys and values in a separate array at the implicit index bucket * 8 + slot
// (Sec. 4.3). On GB300 the unit a random access pays for is one 128-byte L2
// line request: a warp instruction in which four lanes read the four 32-byte
// sectors of one line costs the same as a single 32-byte read. So each bucket
// puts its lookup fields and the entries of its first four slots in one line;
// a key found in slots 0..3 costs one line request, and a negative lookup
// that the filter stops costs one as well.
//
// Line 0, bytes [0, 128):
//   0..15    tag[8]     16-bit tags derived from the primary hash (Sec. 4.3)
//   16..23   bloom      64-bit filter of this bucket's displaced keys (Sec. 4.1)
//   24..27   ctrl       bits 0-7 busy, bits 8-15 in_secondary, bits 16-23 claimed
//                       (set only inside an insert call), bit 31 insert lock
//   28..31   moved      moved counter (Sec. 4.1)
//   tables without timers:          tables with timers (Sec. 4.2):
//   32..95   key[0..3]              32..47   expiry[8] (u16 each)
//   96..127  value[0..3]            48..95   key[0..2]
//                                   96..119  value[0..2], then 8 zero bytes
// Line 1, bytes [128, 256):
//   128..191 key[4..7]              128..207 key[3..7]
//   192..223 value[4..7], then      208..247 value[3..7], then 8 zero bytes
//            32 zero bytes
// With timers the expiries follow the control word, so an insertion decides
// from the first line, an expire scan reads only the first 64 bytes of each
// bucket, and a key found in slots 0..2 is confirmed, tested alive and
// answered from the first line alone.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ckpp {

constexpr uint32_t kSlots = 8;
constexpr uint64_t kHeaderBytes = 256;
constexpr uint32_t kBucketBytes = 256;
constexpr uint32_t kLineBytes = 128;
constexpr uint32_t kMagic = 0x50504B43u;  // "CKPP"
constexpr uint32_t kAbiVersion = 3;       // written to the header; equals CKPP_ABI_VERSION
constexpr uint64_t kSeed2Xor = 0x9E3779B97F4A7C15ull;
constexpr uint32_t kAliveWindow = 1024;   // Sec. 4.2
constexpr uint32_t kMaxStale = 64512;     // Sec. 4.2: 65536 - 1024
constexpr uint32_t kBusyMask = 0xFFu;
constexpr uint32_t kInsecShift = 8;
constexpr uint32_t kClaimShift = 16;  // a slot claimed by an insert, not yet published
constexpr uint32_t kLockBit = 0x80000000u;
constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr uint64_t kMaxBatch = 1ull << 30;
constexpr uint32_t kBatchMaxJobs = 8192;  // jobs per batched launch (prefix sums in shared memory)

// header fields (byte offsets)
constexpr uint32_t kHdrMagic = 0, kHdrAbi = 4, kHdrBuckets = 8, kHdrSlots = 16, kHdrFlags = 20, kHdrSeed = 24,
                   kHdrErr = 32;

// latched device error bits
constexpr uint32_t kErrLockTimeout = 1u;

// per-key status codes (the public contract's values)
constexpr uint8_t kStInserted = 1, kStUpdated = 2, kStFull = 3, kStDeleted = 4, kStNotFound = 5, kStBusy = 6,
                  kStNoTable = 7;

struct TableView {
  uint8_t* buckets;
  uint32_t* err;
  uint64_t nb;
  uint64_t seed;
  uint32_t timers;
  uint32_t pad;
};

struct Key {
  uint64_t k0, k1;
};

struct Addr {
  uint32_t b1, b2;
  uint32_t tag;
  uint64_t bits;  // the two Bloom bits as a mask
};

// ------------------------------------------------------------------ hash
// SplitMix64 output finaliser (Steele, Lea, Flood, OOPSLA 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// H(key, s) = mix(mix(k0 ^ s) ^ k1); k0, k1 = the key's little-endian words.
__device__ __forceinline__ uint64_t hash_key(const Key& k, uint64_t s) { return mix64(mix64(k.k0 ^ s) ^ k.k1); }

// Multiply-shift range reduction of the top 32 bits (Lemire 2019); nb < 2^32.
__device__ __forceinline__ uint32_t reduce(uint64_t h, uint64_t nb) {
  return (uint32_t)(((h >> 32) * (uint64_t)(uint32_t)nb) >> 32);
}

__device__ __forceinline__ Addr address_of(const Key& k, uint64_t nb, uint64_t seed) {
  const uint64_t h1 = hash_key(k, seed);
  const uint64_t h2 = hash_key(k, seed ^ kSeed2Xor);
  Addr a;
  a.b1 = reduce(h1, nb);
  a.b2 = reduce(h2, nb);
  if (a.b2 == a.b1) a.b2 = (a.b1 + 1 == (uint32_t)nb) ? 0u : a.b1 + 1;
  a.tag = (uint32_t)(h1 & 0xFFFF);
  a.bits = (1ull << (h2 & 63)) | (1ull << ((h2 >> 6) & 63));
  return a;
}

// ---------------------------------------------------------- timers (Sec. 4.2)
__device__ __forceinline__ bool alive16(uint32_t expiry, uint32_t now) {
  return (uint32_t)((expiry - now) & 0xFFFFu) < kAliveWindow;
}

// Mask of slots whose 16-bit expiry is alive at now; e0/e1 hold expiry[0..3], [4..7].
__device__ __forceinline__ uint32_t alive_mask(uint64_t e0, uint64_t e1, uint32_t now) {
  uint32_t m = 0;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    m |= (alive16((uint32_t)(e0 >> (16 * s)) & 0xFFFFu, now) ? 1u : 0u) << s;
    m |= (alive16((uint32_t)(e1 >> (16 * s)) & 0xFFFFu, now) ? 1u : 0u) << (s + 4);
  }
  return m;
}

// Mask of slots whose tag equals `tag`; t0/t1 hold tag[0..3], [4..7].
__device__ __forceinline__ uint32_t tag_mask(uint64_t t0, uint64_t t1, uint32_t tag) {
  uint32_t m = 0;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    m |= (((uint32_t)(t0 >> (16 * s)) & 0xFFFFu) == tag ? 1u : 0u) << s;
    m |= (((uint32_t)(t1 >> (16 * s)) & 0xFFFFu) == tag ? 1u : 0u) << (s + 4);
  }
  return m;
}

// ------------------------------------------------------------ addressing
__device__ __forceinline__ uint8_t* bucket_ptr(const TableView& t, uint32_t b) {
  return t.buckets + (uint64_t)b * kBucketBytes;
}
__device__ __forceinline__ uint64_t* bloom_ptr(const TableView& t, uint32_t b) {
  return reinterpret_cast<uint64_t*>(bucket_ptr(t, b) + 16);
}
__device__ __forceinline__ uint32_t* ctrl_ptr(const TableView& t, uint32_t b) {
  return reinterpret_cast<uint32_t*>(bucket_ptr(t, b) + 24);
}
__device__ __forceinline__ uint32_t* moved_ptr(const TableView& t, uint32_t b) {
  return reinterpret_cast<uint32_t*>(bucket_ptr(t, b) + 28);
}
__device__ __forceinline__ uint16_t* tag_ptr(const TableView& t, uint32_t b, uint32_t s) {
  return reinterpret_cast<uint16_t*>(bucket_ptr(t, b)) + s;
}
// The first slot whose entry lives in the second line.
__host__ __device__ constexpr uint32_t first_hi_slot(uint32_t timers) { return timers ? 3u : 4u; }
// Byte offset of a timers table's 8 expiries within a bucket.
constexpr uint32_t kExpiryOff = 32;
// Byte offsets of a slot's key and value within its bucket.
__device__ __forceinline__ uint32_t key_off(uint32_t timers, uint32_t s) {
  if (timers) return s < 3 ? 48u + 16u * s : kLineBytes + 16u * (s - 3);
  return s < 4 ? 32u + 16u * s : kLineBytes + 16u * (s - 4);
}
__device__ __forceinline__ uint32_t value_off(uint32_t timers, uint32_t s) {
  if (timers) return s < 3 ? 96u + 8u * s : 208u + 8u * (s - 3);
  return s < 4 ? 96u + 8u * s : 192u + 8u * (s - 4);
}
__device__ __forceinline__ uint8_t* key_ptr(const TableView& t, uint32_t b, uint32_t s) {
  return bucket_ptr(t, b) + key_off(t.timers, s);
}
__device__ __forceinline__ uint64_t* value_ptr(const TableView& t, uint32_t b, uint32_t s) {
  return reinterpret_cast<uint64_t*>(bucket_ptr(t, b) + value_off(t.timers, s));
}
__device__ __forceinline__ uint16_t* expiry_ptr(const TableView& t, uint32_t b, uint32_t s) {
  return reinterpret_cast<uint16_t*>(bucket_ptr(t, b) + kExpiryOff) + s;
}

// ---------------------------------------------------------- memory access
// Cache policies: L2 evict_first for data read once per lookup (bucket lines
// of a table far larger than L2, streamed keys).
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// 128-bit read-only streaming load.
__device__ __forceinline__ Key ld_key_ro(const void* p, uint64_t pol) {
  Key k;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u64 {%0,%1}, [%2], %3;"
               : "=l"(k.k0), "=l"(k.k1)
               : "l"(p), "l"(pol));
  return k;
}
// Coherent (L2) loads and stores for data other threads modify.
__device__ __forceinline__ void ld256_cg(const void* p, uint64_t (&w)[4]) {
  asm volatile("ld.global.relaxed.gpu.v4.u64 {%0,%1,%2,%3}, [%4];"
               : "=l"(w[0]), "=l"(w[1]), "=l"(w[2]), "=l"(w[3])
               : "l"(p)
               : "memory");
}
__device__ __forceinline__ void ld128_cg(const void* p, uint64_t& a, uint64_t& b) {
  asm volatile("ld.global.relaxed.gpu.v2.u64 {%0,%1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}
__device__ __forceinline__ uint32_t ld32_cg(const void* p) {
  uint32_t v;
  asm volatile("ld.global.relaxed.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t ld64_cg(const void* p) {
  uint64_t v;
  asm volatile("ld.global.relaxed.gpu.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld16_cg(const void* p) {
  uint16_t v;
  asm volatile("ld.global.relaxed.gpu.u16 %0, [%1];" : "=h"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st128_cg(void* p, uint64_t a, uint64_t b) {
  asm volatile("st.global.relaxed.gpu.v2.u64 [%0], {%1,%2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ void st64_cg(void* p, uint64_t v) {
  asm volatile("st.global.relaxed.gpu.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st16_cg(void* p, uint32_t v) {
  asm volatile("st.global.relaxed.gpu.u16 [%0], %1;" ::"l"(p), "h"((uint16_t)v) : "memory");
}

// Set a slot's expiry (timers tables only).
__device__ __forceinline__ void set_expiry(const TableView& t, uint32_t b, uint32_t s, uint32_t expiry) {
  asm volatile("st.global.relaxed.gpu.u16 [%0], %1;" ::"l"(expiry_ptr(t, b, s)), "h"((uint16_t)expiry) : "memory");
}

__device__ __forceinline__ void latch_error(const TableView& t, uint32_t bit) { atomicOr(t.err, bit); }

}  // namespace ckpp
