// Device-side layout, hashing and memory helpers of the GB300 Cuckoo++ table.
//
// HBM layout of one table (caller-owned buffer):
//   [0, 256)             header: magic, geometry copy, latched device error word
//   buckets              n_buckets records of 32 B (64 B with timers), 32 B aligned
//   records              n_buckets * 8 key/value records of 32 B at the implicit
//                        index bucket * 8 + slot (Sec. 4.3 of the paper)
//
// Bucket, first 32-byte sector (everything a lookup reads, Sec. 4.3 "all fields
// accessed when looking up a bucket are in the same cacheline", here the same
// DRAM sector):
//   bytes  0..15  tag[8]   16-bit tags derived from the primary hash
//   bytes 16..23  bloom    64-bit filter of this bucket's displaced keys (Sec. 4.1)
//   bytes 24..27  ctrl     bits 0-7 busy, bits 8-15 in_secondary, bit 31 insert lock
//   bytes 28..31  moved    moved counter (Sec. 4.1)
// With timers, the second sector holds expiry[8] (16-bit, Sec. 4.2) in bytes
// 32..47; bytes 48..63 are reserved (zero).
// Record (32 B, one sector): key (16 B), value (u64), then a u64 whose low 16
// bits copy the slot's expiry in tables with timers (zero otherwise); the
// rest is zero. The bucket's expiry[] is the copy inserts and scans use; the
// record's copy lets a lookup test liveness with the sector it reads anyway.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ckpp {

constexpr uint32_t kSlots = 8;
constexpr uint64_t kHeaderBytes = 256;
constexpr uint32_t kRecordBytes = 32;
constexpr uint32_t kMagic = 0x50504B43u;  // "CKPP"
constexpr uint64_t kSeed2Xor = 0x9E3779B97F4A7C15ull;
constexpr uint32_t kAliveWindow = 1024;   // Sec. 4.2
constexpr uint32_t kMaxStale = 64512;     // Sec. 4.2: 65536 - 1024
constexpr uint32_t kBusyMask = 0xFFu;
constexpr uint32_t kInsecShift = 8;
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

// bounded waits
constexpr int kLockSpins = 1 << 20;

struct TableView {
  uint8_t* buckets;
  uint8_t* records;
  uint32_t* err;
  uint64_t nb;
  uint64_t seed;
  uint32_t bucket_shift;  // log2 of the bucket stride: 5 (32 B) or 6 (64 B, timers)
  uint32_t timers;
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
  return t.buckets + ((uint64_t)b << t.bucket_shift);
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
__device__ __forceinline__ uint16_t* expiry_ptr(const TableView& t, uint32_t b, uint32_t s) {
  return reinterpret_cast<uint16_t*>(bucket_ptr(t, b) + 32) + s;
}
__device__ __forceinline__ uint8_t* record_ptr(const TableView& t, uint32_t b, uint32_t s) {
  return t.records + ((uint64_t)b * kSlots + s) * kRecordBytes;
}

// ---------------------------------------------------------- memory access
// Cache policies: bucket sectors are worth keeping in L2 (the bucket array is
// the table's hot part), records and streamed keys are not.
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// 256-bit read-only load (data not written during the kernel), L1 bypassed.
__device__ __forceinline__ void ld256_ro(const void* p, uint64_t pol, uint64_t (&w)[4]) {
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u64 {%0,%1,%2,%3}, [%4], %5;"
               : "=l"(w[0]), "=l"(w[1]), "=l"(w[2]), "=l"(w[3])
               : "l"(p), "l"(pol));
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
__device__ __forceinline__ void st256_cg(void* p, uint64_t a, uint64_t b, uint64_t c, uint64_t d) {
  asm volatile("st.global.relaxed.gpu.v4.u64 [%0], {%1,%2,%3,%4};" ::"l"(p), "l"(a), "l"(b), "l"(c), "l"(d)
               : "memory");
}
__device__ __forceinline__ void st64_cg(void* p, uint64_t v) {
  asm volatile("st.global.relaxed.gpu.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st16_cg(void* p, uint32_t v) {
  asm volatile("st.global.relaxed.gpu.u16 [%0], %1;" ::"l"(p), "h"((uint16_t)v) : "memory");
}

// Set a slot's expiry: the bucket's copy and the record's copy.
__device__ __forceinline__ void set_expiry(const TableView& t, uint32_t b, uint32_t s, uint32_t expiry) {
  asm volatile("st.global.relaxed.gpu.u16 [%0], %1;" ::"l"(reinterpret_cast<uint16_t*>(t.buckets + ((uint64_t)b << t.bucket_shift) + 32) + s),
               "h"((uint16_t)expiry) : "memory");
  asm volatile("st.global.relaxed.gpu.u16 [%0], %1;" ::"l"(t.records + ((uint64_t)b * kSlots + s) * kRecordBytes + 24),
               "h"((uint16_t)expiry) : "memory");
}

// Records are read as 4 x u64: k0, k1, value, expiry copy (timers) / zero.
__device__ __forceinline__ bool same_key(const uint64_t (&r)[4], const Key& k) { return r[0] == k.k0 && r[1] == k.k1; }

__device__ __forceinline__ void latch_error(const TableView& t, uint32_t bit) { atomicOr(t.err, bit); }

}  // namespace ckpp
