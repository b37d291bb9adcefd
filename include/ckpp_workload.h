/*
 * ckpp_workload.h -- device-side generator of the synthetic 5-tuple traffic
 * (libckpp_workload.so). Not part of the method: it draws the same inputs as
 * paper_1712_09624_gb300/workload.py, bit for bit, directly in device memory,
 * so that workloads of billions of keys need no host generation or upload.
 *
 * Random numbers: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random
 * Numbers: As Easy as 1, 2, 3", SC'11), key (seed, stream); raw output t is word
 * t % 4 of the block for counter t / 4 + 1 (the stream numpy's Philox bit
 * generator produces). Key layout as ckpp_key in ckpp.h.
 *
 * All output pointers are caller-owned device memory; calls are asynchronous
 * on `stream`. Return: 0, or -1 for bad arguments, -2 for a CUDA error.
 */
#ifndef CKPP_WORKLOAD_H
#define CKPP_WORKLOAD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ckpp_wl_stream_t;

/* Keys first .. first+n-1 of the fill of `seed` (workload.fill(seed, m).keys
 * for any m > first+n-1) into out_keys [n][16] (16-byte aligned), and their
 * values (= index) into out_vals [n] if not NULL. */
int ckpp_wl_fill_keys(uint64_t seed, uint64_t first, uint64_t n, uint8_t* out_keys, uint64_t* out_vals,
                      ckpp_wl_stream_t stream);

/* Fill keys at arbitrary indices: out_keys[i] = key idx[i] of the fill of `seed`
 * (idx: device uint64 [n]). */
int ckpp_wl_keys_at(uint64_t seed, const uint64_t* idx, uint64_t n, uint8_t* out_keys, ckpp_wl_stream_t stream);

/* workload.lookup_batch(seed, n, workload.fill(seed, n_inserted), neg_rate,
 * batch_id): keys [n][16], expected found flags [n] and values [n] (either
 * expectation pointer may be NULL). */
int ckpp_wl_lookup_batch(uint64_t seed, uint64_t batch_id, uint64_t n, uint64_t n_inserted, double neg_rate,
                         uint8_t* out_keys, uint8_t* expect_found, uint64_t* expect_value, ckpp_wl_stream_t stream);

/* L2 read probe (measurement): `passes` streaming reads of buf (`bytes` a
 * multiple of 16, 16-byte aligned device memory; a buffer smaller than L2 is
 * read from L2 after the first pass) with 16-byte ld.global.cg loads, one
 * grid of 8 blocks of 256 threads per SM. sink: device uint64 the loads feed
 * (left unchanged in practice). Bytes read = bytes x passes; time it with
 * events on `stream`. Returns 0, -1 (bad argument) or -2. */
int ckpp_wl_l2_read(const uint8_t* buf, uint64_t bytes, uint32_t passes, uint64_t* sink, ckpp_wl_stream_t stream);

/* Host-link probe (measurement): the host I/O of a lookup on host buffers,
 * without a table. keys [n][16] (16-byte aligned), out_vals [n] (8-byte
 * aligned) and out_found [n] may be pinned host or device memory; for each i,
 * with k0, k1 the key's two little-endian 64-bit words, out_vals[i] =
 * k0 ^ (k1 << 1) and out_found[i] = k1 & 1. Each lane reads one key and each
 * warp writes its 32 results as 16-byte vectors when both outputs are 16-byte
 * aligned. Returns 0, -1 (bad argument) or -2. */
int ckpp_wl_host_io(const uint8_t* keys, uint64_t n, uint64_t* out_vals, uint8_t* out_found,
                    ckpp_wl_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* CKPP_WORKLOAD_H */
