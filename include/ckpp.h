/*
 * ckpp.h -- C ABI of the GB300 Cuckoo++ flow-table library (libckpp.so).
 *
 * The method is Cuckoo++ (Le Scouarnec, "Cuckoo++ Hash Tables: High-Performance
 * Hash Tables for Networking Applications", 2017): a bucketized two-choice
 * cuckoo hash table of 8-slot buckets whose primary bucket carries a 64-bit
 * Bloom filter of the keys displaced to their secondary bucket (Sec. 4.1), with
 * optional 16-bit expiration timers (Sec. 4.2).
 *
 * Conventions shared by every call below:
 *  - All array arguments are DEVICE pointers owned by the caller (e.g. torch
 *    tensors); the library never frees them. The table handle is host memory
 *    owned by the library (ckpp_create / ckpp_destroy).
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and never synchronise the device, except ckpp_stats and
 *    ckpp_sync_status, which say so.
 *  - Return value: CKPP_OK (0) or a negative CKPP_E* code. A call that returns an
 *    error launched nothing. Per-key outcomes go to status arrays, never to the
 *    return value.
 *  - Errors found on the device (a bounded wait that gave up) are latched in the
 *    table's device status word; ckpp_sync_status reads and clears it.
 *  - Calls on one table must be ordered (one stream, or events): the table is a
 *    single-writer structure, as in the paper's share-nothing setting (Sec. 2).
 *  - Batches hold at most 2^32 - 1 keys.
 *  - Timers: with CKPP_TIMERS, `now` is the caller's time in quantised units
 *    (Sec. 4.2, e.g. 30 s); an entry inserted with ttl expires after now + ttl
 *    and is alive iff (uint16)(expiry - now) < 1024, so ttl <= 1023. A full
 *    ckpp_expire scan must run at least every 64512 units; a call whose `now` is
 *    more than 64512 units past the last scan (or the first timed call) returns
 *    CKPP_ESTALE. Without CKPP_TIMERS, now/ttl/refresh_ttl are ignored.
 */
#ifndef CKPP_H
#define CKPP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t without including the CUDA runtime headers. */
typedef struct CUstream_st* ckpp_stream_t;

#define CKPP_ABI_VERSION 3

/* return codes */
#define CKPP_OK 0
#define CKPP_EINVAL (-1)  /* bad geometry, NULL or misaligned pointer, buffer too small, n too large */
#define CKPP_ECUDA (-2)   /* a CUDA launch or runtime call failed */
#define CKPP_ESTALE (-3)  /* `now` is more than 64512 units past the last expire scan */
#define CKPP_EBUSY (-4)   /* a bounded device wait gave up (latched; see ckpp_sync_status) */

/* per-key status codes (uint8) */
#define CKPP_ST_INSERTED 1  /* the key had no live entry; it now has one            */
#define CKPP_ST_UPDATED 2   /* the key had a live entry; value and expiry replaced  */
#define CKPP_ST_FULL 3      /* no free slot and no cuckoo path found; table unchanged for this key */
#define CKPP_ST_DELETED 4   /* the key had a live entry; it is gone                 */
#define CKPP_ST_NOT_FOUND 5 /* the key had no live entry                            */
#define CKPP_ST_BUSY 6      /* a bounded lock wait gave up; the key was not processed */
#define CKPP_ST_NO_TABLE 7  /* batch calls: the key's table index names no table of the batch */

/* geometry flags */
#define CKPP_TIMERS 1u

/* A 5-tuple flow key: 16 bytes, 16-byte aligned in arrays, little endian,
 * pad bytes must be zero (they are hashed and compared like the rest). */
typedef struct ckpp_key {
  uint32_t src_ip;
  uint32_t dst_ip;
  uint16_t src_port;
  uint16_t dst_port;
  uint8_t proto;
  uint8_t pad[3];
} ckpp_key;

/* Table geometry. n_buckets in [2, 2^32 - 1]; slots_per_bucket must be 8
 * (Sec. 4.3: 8 16-bit tags per bucket); flags: CKPP_TIMERS or 0; seed selects
 * the hash functions. */
typedef struct ckpp_geometry {
  uint64_t n_buckets;
  uint32_t slots_per_bucket;
  uint32_t flags;
  uint64_t seed;
} ckpp_geometry;

typedef struct ckpp_table ckpp_table;

/* Table statistics (Fig. 2, Fig. 5 and Table 2 of the paper are built from these). */
typedef struct ckpp_stats {
  uint64_t n_buckets;
  uint64_t n_slots;
  uint64_t n_occupied;      /* busy slots, alive or dead                          */
  uint64_t n_live;          /* busy and alive at `now`                            */
  uint64_t n_in_secondary;  /* busy slots whose entry sits in its secondary bucket */
  uint64_t n_moved_zero;    /* buckets whose moved counter is 0                   */
  uint64_t moved_sum;       /* sum of moved counters (= n_in_secondary)           */
  uint64_t bloom_bits_set;  /* total set bits over all filters                    */
  uint64_t bloom_pop_sq;    /* sum over buckets of popcount(filter)^2             */
  uint64_t moved_hist[16];  /* buckets with moved counter c (c = 15: 15 or more)  */
} ckpp_stats;

/* Bytes of device memory a table of this geometry needs (0 if the geometry is
 * invalid): a 256-byte header, then n_buckets buckets of 256 bytes. A bucket
 * is two 128-byte lines. Line 0 holds the fields a lookup reads first (8
 * 16-bit tags, the 64-bit filter, the busy / in_secondary / claimed / lock word and the
 * moved counter; Sec. 4.1, 4.3) with the keys and values of slots 0..3, or,
 * with CKPP_TIMERS, of slots 0..2 and the 8 16-bit expiries (Sec. 4.2). Line 1
 * holds the keys and values of the other slots. The keys and values of a
 * bucket's slots thus sit in the bucket itself rather than in a separate array
 * at the implicit index of Sec. 4.3: a random access costs one 128-byte line
 * on this GPU, whatever part of the line it uses. */
size_t ckpp_required_bytes(const ckpp_geometry* geometry);

/* Device workspace bytes an insert or delete batch of n keys needs (scratch for
 * resolving in-batch duplicate keys and for the displacement passes). Once an
 * insert call has completed on its stream, the first 32 bytes of its workspace
 * hold diagnostics as uint32 words: [0] keys that found no free or dead slot in
 * either bucket, [3] of those, keys the one-move pass left, [5] keys the grid
 * search left, [6] keys the second search pass left (the last pass reports the
 * ones it cannot place FULL). The other words are scratch. */
size_t ckpp_workspace_bytes(uint64_t n);

/* Create a table in the caller's device buffer dev_buf (at least
 * ckpp_required_bytes, 256-byte aligned) and clear it on `stream`. The buffer
 * must outlive the handle and stay untouched by the caller. On success *out
 * receives a host handle. Errors: CKPP_EINVAL (geometry, NULL, size, alignment),
 * CKPP_ECUDA. */
int ckpp_create(ckpp_table** out, const ckpp_geometry* geometry, void* dev_buf, size_t bytes,
                ckpp_stream_t stream);

/* Release the host handle. Does not free dev_buf and does not synchronise: the
 * caller must not reuse dev_buf before the table's queued work has finished. */
int ckpp_destroy(ckpp_table* table);

/* Open a table whose bytes already sit in dev_buf: a buffer a table was
 * created in, or a copy of one (checkpoint and resume: a table is its buffer,
 * so saving it is one device-to-host copy of ckpp_required_bytes bytes, taken
 * while no call on the table is running, and restoring it is the copy back
 * plus this call; no counterpart in the paper). Reads the 256-byte header on
 * `stream` and synchronises it, checks the magic, the ABI version and the
 * geometry (8 slots, known flags, n_buckets in range, bytes at least the
 * geometry's size), and returns a handle over the buffer without touching the
 * buckets; the latched device error word is kept. `now` restarts the
 * staleness clock of a timers table (Sec. 4.2: a timed call more than 64512
 * units after it returns CKPP_ESTALE): pass the time of the table's last expire
 * scan, or an earlier one. dev_buf must stay untouched by the caller and
 * outlive the handle, as for ckpp_create. Errors: CKPP_EINVAL (NULL,
 * misaligned, too small, not a table of this ABI version), CKPP_ECUDA. */
int ckpp_attach(ckpp_table** out, void* dev_buf, size_t bytes, uint32_t now, ckpp_stream_t stream);

/* Batched lookup (Sec. 2, Sec. 4.1 and Fig. 4): for every key i, read the primary
 * bucket, compare tags, confirm the full key against the matching slot's key;
 * on a miss test the two Bloom bits of the primary's filter and read the
 * secondary bucket only if both are set. With timers dead entries are ignored (Sec. 4.2) and,
 * if refresh_ttl > 0, a hit sets the entry's expiry to now + refresh_ttl.
 *   keys      [n] ckpp_key, 16-byte aligned
 *   out_vals  [n] uint64, 8-byte aligned: the value, or 0 on a miss
 *   out_found [n] uint8: 1 on a hit, 0 on a miss
 * Unlike the other calls, keys / out_vals / out_found may also be pinned host
 * memory (cudaHostAlloc or cudaHostRegister): the kernel then reads the keys
 * and writes the results in place over the host link (NVLink-C2C on GB300),
 * with no staging copy; the caller must not touch them until the stream
 * reaches the call's completion. Pageable host memory is rejected (EINVAL).
 * Errors: CKPP_EINVAL, CKPP_ESTALE, CKPP_ECUDA. */
int ckpp_bulk_lookup(ckpp_table* table, const ckpp_key* keys, uint64_t n, uint64_t* out_vals,
                     uint8_t* out_found, uint32_t now, uint16_t refresh_ttl, ckpp_stream_t stream);

/* Lookup strategies. CKPP_LOOKUP_BLOOM is Cuckoo++ (Sec. 4.1) and what
 * ckpp_bulk_lookup does; the other two are the strategies of Sec. 3 on the same
 * table, kept for measuring what the filter saves: OPTIMISTIC reads the
 * secondary bucket after every primary miss, PESSIMISTIC reads both buckets of
 * every key. All three return identical results. */
#define CKPP_LOOKUP_BLOOM 0
#define CKPP_LOOKUP_OPTIMISTIC 1
#define CKPP_LOOKUP_PESSIMISTIC 2

/* ckpp_bulk_lookup with an explicit strategy (device buffers only).
 * Errors: CKPP_EINVAL (also for an unknown variant), CKPP_ESTALE, CKPP_ECUDA. */
int ckpp_bulk_lookup_variant(ckpp_table* table, const ckpp_key* keys, uint64_t n, uint64_t* out_vals,
                             uint8_t* out_found, uint32_t now, uint16_t refresh_ttl, int variant,
                             ckpp_stream_t stream);

/* ---- Batched form: many tables, one launch --------------------------------
 * One persistent kernel serves the lookup jobs of many independent tables (the
 * GPU counterpart of the paper's one private table per core, Sec. 2 and 5.3).
 * Jobs live in device memory and may change between launches, so the launch can
 * be captured in a CUDA graph once and replayed. */
#define CKPP_BATCH_MAX_JOBS 8192

typedef struct ckpp_lookup_job {
  const ckpp_key* keys; /* device, 16-byte aligned, n keys */
  uint64_t* out_vals;   /* device, n values (0 on a miss) */
  uint8_t* out_found;   /* device, n flags */
  uint32_t n;           /* keys in this job (0 allowed) */
  uint32_t table;       /* index into the batch's table list; jobs naming no table are skipped */
} ckpp_lookup_job;

/* Kernel configuration. threads_per_key: 1, 2 or 4 lanes of a warp per key
 * in one iteration, so 32 / threads_per_key lanes own keys and every lane
 * helps fetch their bucket lines (each 128-byte line is copied by 8 lanes of
 * 16 bytes, four lines per warp instruction, one line request each).
 * keys_per_warp: 0 (derived) or 32 / threads_per_key. group_depth: 1 or 2
 * keys owned per owning lane, i.e. up to 32 / threads_per_key x group_depth
 * line requests a warp has in flight. blocks_per_sm: 1..4 persistent blocks
 * of 512 threads per SM. A NULL tuning is {1, 1, 2, 32}. */
typedef struct ckpp_batch_tuning {
  uint32_t threads_per_key;
  uint32_t group_depth;
  uint32_t blocks_per_sm;
  uint32_t keys_per_warp;
} ckpp_batch_tuning;

typedef struct ckpp_batch ckpp_batch;

/* Device bytes of a batch descriptor for n_tables tables (their views and a
 * 256-byte control block the lookup kernel uses to hand out work; lookups that
 * use one descriptor must therefore be ordered, e.g. on one stream). */
size_t ckpp_batch_bytes(uint32_t n_tables);

/* Describe tables[0..n_tables) (handles of tables on the current device) in
 * dev_buf (>= ckpp_batch_bytes, 256-byte aligned, caller-owned) on `stream`.
 * The tables must outlive the batch. Errors: CKPP_EINVAL, CKPP_ECUDA. */
int ckpp_batch_create(ckpp_batch** out, ckpp_table* const* tables, uint32_t n_tables, void* dev_buf, size_t bytes,
                      ckpp_stream_t stream);

/* Release the host handle (dev_buf stays the caller's). */
int ckpp_batch_destroy(ckpp_batch* batch);

/* Insert (as ckpp_bulk_insert) keys bound for many tables of a batch in one
 * call: key i goes to the batch's table table_ids[i] (device uint32 [n]); the
 * same key bound for two tables is two keys. Statuses as ckpp_bulk_insert, plus
 * CKPP_ST_NO_TABLE for an index beyond the batch's tables. Workspace as for
 * ckpp_bulk_insert (ckpp_workspace_bytes(n)). Errors: CKPP_EINVAL, CKPP_ESTALE
 * (a timers table), CKPP_ECUDA. */
int ckpp_batch_insert(ckpp_batch* batch, const ckpp_key* keys, const uint32_t* table_ids, const uint64_t* vals,
                      uint64_t n, uint32_t now, uint16_t ttl, uint8_t* status, void* workspace,
                      size_t workspace_bytes, ckpp_stream_t stream);

/* Delete (as ckpp_bulk_delete) keys of many tables of a batch in one call;
 * key i belongs to table table_ids[i]. Errors as ckpp_batch_insert. */
int ckpp_batch_delete(ckpp_batch* batch, const ckpp_key* keys, const uint32_t* table_ids, uint64_t n, uint32_t now,
                      uint8_t* status, void* workspace, size_t workspace_bytes, ckpp_stream_t stream);

/* Look up every job's keys in its table (filter-pruned, as ckpp_bulk_lookup,
 * without refresh) in one launch. d_jobs: device array of at least max_jobs
 * jobs; d_n_jobs: NULL (use max_jobs) or a device uint32 job count, clamped to
 * max_jobs. tuning: NULL for the default (see ckpp_batch_tuning). Launches on
 * one batch must not overlap on the GPU (they share its work counter). The job data is not validated on the host: every job's pointers must
 * be valid device memory. The launch draws work from counters in the
 * descriptor, so lookups on one descriptor must not run concurrently (order
 * them on one stream; use a second descriptor over the same tables for a
 * second stream). Errors: CKPP_EINVAL (max_jobs above CKPP_BATCH_MAX_JOBS, bad
 * tuning), CKPP_ESTALE (a timers table), CKPP_ECUDA. */
int ckpp_batch_lookup(ckpp_batch* batch, const ckpp_lookup_job* d_jobs, uint32_t max_jobs, const uint32_t* d_n_jobs,
                      uint32_t now, const ckpp_batch_tuning* tuning, ckpp_stream_t stream);

/* Batched insert-or-update (Sec. 2 cuckoo insertion; Sec. 4.1 filter and moved
 * counter upkeep, including moves along a cuckoo path; Sec. 4.2 dead slots are
 * reused as free). The batch has the result of inserting keys one by one in
 * index order: the last occurrence of a key supplies its value, the first
 * occurrence reports INSERTED or UPDATED and later ones UPDATED. A key that finds
 * no slot and no cuckoo path reports FULL (every occurrence) and leaves the table
 * unchanged for that key.
 *   keys   [n] ckpp_key, 16-byte aligned;  vals [n] uint64, 8-byte aligned
 *   status [n] uint8 out: CKPP_ST_INSERTED / UPDATED / FULL / BUSY
 *   ttl    expiry = now + ttl, ttl <= 1023 (timers only)
 *   workspace: device memory of at least ckpp_workspace_bytes(n) bytes,
 *   256-byte aligned, used only while the call's work runs on `stream`.
 * Errors: CKPP_EINVAL, CKPP_ESTALE, CKPP_ECUDA. */
int ckpp_bulk_insert(ckpp_table* table, const ckpp_key* keys, const uint64_t* vals, uint64_t n,
                     uint32_t now, uint16_t ttl, uint8_t* status, void* workspace, size_t workspace_bytes,
                     ckpp_stream_t stream);

/* How insert calls (ckpp_bulk_insert, ckpp_batch_insert, the no-alloc insert)
 * launch their work; no counterpart in the paper, and the results are the
 * same either way. Modes:
 *   CKPP_INSERT_LAUNCH_CHAIN   (the default) a chain of dependent kernels:
 *                              duplicate resolution, the slot claims, their
 *                              publication, the one-move pass, three
 *                              cuckoo-path searches, the filter fixup, each
 *                              launched to start while its predecessor drains;
 *   CKPP_INSERT_LAUNCH_SINGLE  one cooperative launch running the same stages
 *                              separated by grid-wide barriers, sized to the
 *                              batch, with stages that have nothing to do
 *                              skipped (a device without cooperative launch
 *                              uses the chain).
 * Measured on GB300 the two take the same time within a few percent at every
 * batch size (a 1-key call about 35 us, a 64K-key call about 105 us at load
 * factor 0.8): the stages' dependent memory round trips, not the launches,
 * set it.
 * The mode is process-wide; set it while no insert call is being issued.
 * Returns the previous mode, or CKPP_EINVAL for an unknown one. */
#define CKPP_INSERT_LAUNCH_CHAIN 0
#define CKPP_INSERT_LAUNCH_SINGLE 1
int ckpp_set_insert_launch(int mode);

/* Batched delete (Sec. 4.1: deleting a key stored in its secondary bucket
 * decrements the primary's moved counter and resets the filter at zero). The
 * first occurrence of a key in the batch reports DELETED if it had a live entry,
 * every other occurrence NOT_FOUND. A dead entry of the key is removed as well.
 *   keys [n] ckpp_key, 16-byte aligned;  status [n] uint8 out
 *   workspace as for ckpp_bulk_insert.
 * Errors: CKPP_EINVAL, CKPP_ESTALE, CKPP_ECUDA. */
int ckpp_bulk_delete(ckpp_table* table, const ckpp_key* keys, uint64_t n, uint32_t now, uint8_t* status,
                     void* workspace, size_t workspace_bytes, ckpp_stream_t stream);

/* Largest batch ckpp_bulk_insert_noalloc accepts. */
#define CKPP_NOALLOC_MAX_KEYS 65536

/* Bulk insert for callers that cannot allocate device memory. No counterpart
 * in the paper: it is ckpp_bulk_insert with the same semantics, arguments and
 * status codes, minus the workspace. Its scratch is a fixed device array built
 * into libckpp.so (about 6 MB, enough for CKPP_NOALLOC_MAX_KEYS keys), which
 * every GPU that loads the library holds until the process exits. It suits
 * callers that own no allocator when they insert: a data-plane thread that must
 * never call cudaMalloc/cudaFree (cudaFree can stall the whole device), or a
 * plugin whose host framework owns all device memory.
 *  - n > CKPP_NOALLOC_MAX_KEYS returns CKPP_EINVAL (split the batch).
 *  - The call allocates nothing: no cudaMalloc, cudaFree or allocating library
 *    routine. It clears the parts of the array that must start at zero.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture. Call with the table's device current. The
 *    address is kept for the life of the process: after cudaDeviceReset,
 *    reload libckpp.so before calling again.
 *  - All calls share the one array: calls whose work overlaps on the GPU
 *    (different streams, or several tables at once) race and corrupt each
 *    other's results. Order them on one stream or with events.
 * Errors: CKPP_EINVAL, CKPP_ESTALE, CKPP_ECUDA. */
int ckpp_bulk_insert_noalloc(ckpp_table* table, const ckpp_key* keys, const uint64_t* vals, uint64_t n,
                             uint32_t now, uint16_t ttl, uint8_t* status, ckpp_stream_t stream);

/* ---- Hash sharding: one table split over several GPUs ---------------------
 * Each rank owns the keys of its shard in a table of its own (the paper's
 * private per-core tables, Sec. 2 and Sec. 5.3, with the keys partitioned by
 * hash instead of by core). A bulk call over the whole table partitions its
 * batch by owner (ckpp_shard_partition), sends each part to its owner (an
 * all-to-all, outside this library), runs the owner's ordinary bulk call,
 * sends the results back (a second all-to-all) and writes them in the
 * caller's order (ckpp_shard_unpermute). The shard of a key is
 *   ((H1 >> 16) & 0xFFFF) * n_shards >> 16,
 * bits 16-31 of the primary hash, which neither the tag (bits 0-15) nor the
 * primary bucket (bits 32-63) uses, so each shard's table sees uniform buckets
 * and tags. H1 is the table's primary hash with the given seed. */
#define CKPP_MAX_SHARDS 64

/* Device workspace bytes of ckpp_shard_partition (0 if n or n_shards is out
 * of range). */
size_t ckpp_shard_workspace_bytes(uint64_t n, uint32_t n_shards);

/* Stable partition of a batch by shard (n_shards in [1, CKPP_MAX_SHARDS]).
 *   keys      [n] ckpp_key, 16-byte aligned;  vals [n] uint64 or NULL
 *   out_pos   [n] uint32: the sorted position of each key of the batch (written
 *             in batch order; ckpp_shard_unpermute reads it the same way)
 *   out_keys  [n] ckpp_key (16-byte aligned), out_vals [n] uint64 (NULL iff
 *             vals is NULL): keys and values in sorted order, i.e. shard 0's
 *             keys first, each shard's keys in batch order
 *   out_counts [n_shards] uint64: keys per shard
 *   workspace: ckpp_shard_workspace_bytes(n, n_shards) device bytes.
 * All device pointers, caller-owned; asynchronous on `stream`.
 * Errors: CKPP_EINVAL, CKPP_ECUDA. */
int ckpp_shard_partition(const ckpp_key* keys, const uint64_t* vals, uint64_t n, uint64_t seed, uint32_t n_shards,
                         uint32_t* out_pos, ckpp_key* out_keys, uint64_t* out_vals, uint64_t* out_counts,
                         void* workspace, size_t workspace_bytes, ckpp_stream_t stream);

/* Bring results that arrive in sorted order back to the caller's order:
 * out[i] = in[pos[i]] for i < n (pos: ckpp_shard_partition's out_pos), for a
 * uint64 array (in_u64/out_u64, both or neither) and a uint8 array
 * (in_u8/out_u8, both or neither). The outputs are written in batch order.
 * Device pointers, caller-owned. Errors: CKPP_EINVAL, CKPP_ECUDA. */
int ckpp_shard_unpermute(const uint32_t* pos, uint64_t n, const uint64_t* in_u64, const uint8_t* in_u8,
                         uint64_t* out_u64, uint8_t* out_u8, ckpp_stream_t stream);

/* Expiration scan (Sec. 4.2): delete every dead entry of every bucket, with
 * moved-counter upkeep, and record `now` as the last scan time. If
 * d_n_expired is not NULL, the number of deleted entries is ADDED to the
 * device uint64 it points to. No-op scan (but the time is recorded) without
 * timers. Errors: CKPP_EINVAL, CKPP_ECUDA. */
int ckpp_expire(ckpp_table* table, uint32_t now, uint64_t* d_n_expired, ckpp_stream_t stream);

/* Table statistics at time `now`, written to host memory. Synchronises
 * `stream`. Errors: CKPP_EINVAL, CKPP_ECUDA. */
int ckpp_stats_get(ckpp_table* table, uint32_t now, ckpp_stats* host_out, ckpp_stream_t stream);

/* For a lookup batch, count the memory reads a lookup strategy (variant, see
 * ckpp_bulk_lookup_variant) makes without performing the lookup (no refresh):
 * d_counts[0] += primary bucket reads (n), d_counts[1] += secondary bucket
 * reads, d_counts[2] += key/value record reads (tag-matching candidates,
 * examined in slot order until the key is met, Sec. 2), d_counts[3] += second-
 * line reads (a bucket's line 1, read when a candidate or, with timers, the
 * value lies there). d_counts is a device uint64[4]. The first three state a
 * batch's algorithmic bytes; d_counts[0] + d_counts[1] + d_counts[3] is the
 * number of 128-byte line requests the lookup makes.
 * Errors: CKPP_EINVAL, CKPP_ESTALE, CKPP_ECUDA. */
int ckpp_lookup_probe_counts(ckpp_table* table, const ckpp_key* keys, uint64_t n, uint32_t now, int variant,
                             uint64_t* d_counts, ckpp_stream_t stream);

/* Synchronise `stream`, then read and clear the table's latched device error
 * word: CKPP_OK, or CKPP_EBUSY if a bounded wait gave up since the last call.
 * Errors: CKPP_EINVAL, CKPP_ECUDA. */
int ckpp_sync_status(ckpp_table* table, ckpp_stream_t stream);

/* Geometry of an existing table (host copy). Errors: CKPP_EINVAL. */
int ckpp_get_geometry(const ckpp_table* table, ckpp_geometry* out);

/* Time of the last expire scan (or first timed call) and whether one was set. */
int ckpp_get_last_scan(const ckpp_table* table, uint32_t* last_scan, int* have_epoch);

/* Static text for a return code. */
const char* ckpp_error_string(int code);

/* CKPP_ABI_VERSION of the loaded library. */
int ckpp_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CKPP_H */
