/*
 * ckpp_serve.h -- host-side runtime of the served form (libckpp.so).
 *
 * The served form answers a stream of packet bursts, each a lookup of flows or
 * an insert of new flows on one of many tables, the way the paper's per-core
 * flow tables see traffic (Sec. 2: packets are processed in batches, and a
 * flow's packets are looked up after the flow is inserted). The device work is
 * the batched calls of ckpp.h; this header is the host policy that turns the
 * arrival stream into launches: which bursts go out in which launch, and when.
 *
 * The planner and the job staging are plain host code: no CUDA call, no device
 * memory, usable without a GPU; their pointers are host pointers owned by the
 * caller. The serving loops at the end drive the device through ckpp.h.
 *
 * The turn planner. Called whenever the caller's loop is free to launch, it
 * plans one turn:
 *  - admission: every burst that has arrived by `now`, in arrival order, while
 *    the staging footprint (bytes_per_key x keys) of the bursts admitted and not
 *    yet completed stays within footprint_bytes; a burst that does not fit
 *    waits, and a burst larger than the whole budget is admitted alone once
 *    nothing else is outstanding;
 *  - lookups: the admitted lookup bursts go out in this turn;
 *  - write coalescing: admitted insert bursts wait and go out together (one
 *    multi-table insert over a contiguous range of the caller's insert pool)
 *    once insert_flush_keys keys wait, the oldest waited insert_flush_s, a
 *    lookup held behind them waited lookup_hold_s, the stream ended, or the
 *    waiting inserts hold budget that a newly arrived burst needs;
 *  - per-table arrival order: on every table, lookups and inserts take effect
 *    in arrival order, so each lookup sees exactly the inserts of its table
 *    that arrived before it. A turn launches, in this order, the lookups whose
 *    table has no waiting insert; the flush of the waiting inserts; the lookups
 *    that arrived while an insert of their table was waiting (held until that
 *    flush). An insert that arrives for a table with a held lookup ends the
 *    turn's admission and forces the flush (the held lookup must not see it).
 *    A lookup beyond max_jobs ends admission too, and forces the flush of any
 *    waiting inserts.
 *  - overlap (optional): flushes run on a second stream, beside later turns'
 *    lookups. A turn then launches its free lookups on the first stream and,
 *    on the second, after waiting for them: the lookups whose table has a
 *    flush in flight (launched, not yet reported complete: "trailing", so
 *    they still see every earlier insert of their table), the flush, and the
 *    lookups held behind it. A trailing lookup runs before the turn's own
 *    flush, which holds only inserts that arrived after it.
 */
#ifndef CKPP_SERVE_H
#define CKPP_SERVE_H

#include <stddef.h>
#include <stdint.h>

#include "ckpp.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ckpp_planner ckpp_planner;

typedef struct ckpp_plan_config {
  double insert_flush_s;       /* flush once the oldest waiting insert waited this long (s) */
  double lookup_hold_s;        /* ... or a lookup held behind them waited this long (s) */
  uint64_t insert_flush_keys;  /* ... or this many insert keys wait */
  uint64_t footprint_bytes;    /* staging budget of admitted, uncompleted bursts */
  uint64_t bytes_per_key;      /* staging footprint of one key (keys in, results out) */
  uint32_t max_jobs;           /* lookup bursts per turn (all its lookup launches together), >= 1 */
  uint32_t overlap;            /* 1: flushes on a second stream (see above); 0: one stream */
} ckpp_plan_config;

/* The stream, in arrival order (arrival nondecreasing; checked). n bursts:
 *   arrival [n] seconds since the start;  table [n] target table (< 2^20)
 *   size    [n] keys in the burst;        insert [n] 1 = insert of new flows, 0 = lookup
 *   offset  [n] inserts: first key in the insert pool (inserts' ranges follow one another in
 *               arrival order); lookups: the caller's own offset (passed through to staging)
 * The arrays are borrowed, not copied: they must outlive the planner.
 * Errors: CKPP_EINVAL (NULL pointer, n < 0, unsorted arrival, table out of range, bad config). */
int ckpp_plan_create(const double* arrival, const uint32_t* table, const uint32_t* size, const uint8_t* insert,
                     const int64_t* offset, int64_t n, const ckpp_plan_config* cfg, ckpp_planner** out);
int ckpp_plan_destroy(ckpp_planner* p);

#define CKPP_PLAN_IDLE 0    /* nothing to do before host time turn->wake */
#define CKPP_PLAN_BLOCK 1   /* the budget is full: wait for the oldest outstanding turn */
#define CKPP_PLAN_NONE 2    /* bursts were admitted, nothing to launch yet */
#define CKPP_PLAN_LAUNCH 3  /* launch the turn */

typedef struct ckpp_turn {
  int32_t action;        /* CKPP_PLAN_* */
  int32_t pad;
  double wake;           /* IDLE: host time of the next arrival or flush deadline */
  int64_t admitted_lo;   /* bursts admitted by this call: [admitted_lo, admitted_hi) */
  int64_t admitted_hi;
  int64_t n_lookups;     /* bursts written to lookups[] (first lookup launch) */
  int64_t n_inserts;     /* bursts written to inserts[] (the flush; 0 = no flush) */
  int64_t n_after;       /* bursts written to after[] (lookups held behind the flush) */
  int64_t insert_first;  /* insert-pool offset of inserts[0] */
  int64_t insert_keys;   /* keys of inserts[] (a contiguous range of the insert pool) */
  int64_t nbytes;        /* footprint the turn's bursts release when it completes (with overlap: its
                            first-stream part, the free lookups) */
  int64_t n_trailing;    /* overlap: bursts written to trailing[] (lookups behind a flush in flight) */
  int64_t nbytes_b;      /* overlap: footprint of the second-stream part (trailing, flush, held) */
} ckpp_turn;

/* Plans one turn at host time `now`; `outstanding` != 0 when an earlier turn
 * has not completed. lookups/trailing/inserts/after receive burst indices
 * (ascending) and must each hold `cap` entries (trailing may be NULL without
 * overlap); cap >= n always suffices.
 * Errors: CKPP_EINVAL (NULL pointer, cap too small for the turn: the planner's
 * state is then unchanged). */
int ckpp_plan_next(ckpp_planner* p, double now, int outstanding, ckpp_turn* turn, int64_t* lookups,
                   int64_t* trailing, int64_t* inserts, int64_t* after, int64_t cap);
/* Reports a launched turn (with overlap: its first-stream part) as completed:
 * frees its footprint (turn->nbytes). */
int ckpp_plan_complete(ckpp_planner* p, int64_t nbytes);
/* Overlap: reports a turn's second-stream part as completed (parts complete
 * in launch order): frees turn->nbytes_b and, if the part carried a flush
 * (flushed != 0), ends that flush's flight on its tables. */
int ckpp_plan_complete_b(ckpp_planner* p, int64_t nbytes_b, int flushed);
/* The planner's state: insert keys waiting, footprint outstanding, and whether
 * every burst has been admitted and launched. Any output pointer may be NULL. */
int ckpp_plan_state(const ckpp_planner* p, int64_t* pending_keys, int64_t* flight_bytes, int* finished);

/* Writes one ckpp_lookup_job (ckpp.h) per burst bursts[i]: keys at
 * pool_keys[t] + 16 * offset[b], out_vals at pool_vals[t] + 8 * offset[b],
 * out_found at pool_found[t] + offset[b], n = size[b], table = t, with
 * t = table[b]. The pool addresses are the caller's (device) buffers, used as
 * numbers only. jobs: host memory for n_bursts records (32 bytes each).
 * Errors: CKPP_EINVAL (NULL pointer, n_bursts < 0). */
int ckpp_serve_stage_jobs(const int64_t* bursts, int64_t n_bursts, const uint32_t* table, const int64_t* offset,
                          const uint32_t* size, const uint64_t* pool_keys, const uint64_t* pool_vals,
                          const uint64_t* pool_found, void* jobs);

/* ------------------------------------------------------------------------
 * The serving loops. They run a whole stream in real time on the host, on one
 * CUDA stream, and return when every burst has completed. Host time starts at
 * the call; a burst is admitted once its arrival time has passed.
 *
 * ckpp_serve_run (continuous batching) asks the planner for a turn whenever it
 * is free to launch and, without waiting for earlier turns, stages the turn's
 * lookup jobs in a pinned ring buffer, copies them to the device job array and
 * launches, in this order: ckpp_batch_lookup over the lookups whose table has
 * no waiting insert; ckpp_batch_insert over the flushed inserts (one
 * contiguous range of the insert pool, `now` 0, ttl 0); ckpp_batch_lookup over
 * the lookups held behind them. A turn completes when an event recorded after
 * its launches does; its bursts then release their footprint.
 *
 * With the planner's overlap mode, ckpp_serve_run puts each turn's free lookups
 * on `stream` and its trailing lookups, flush and held lookups on a second
 * stream it creates, which waits for the first at each turn; it keeps at most
 * max_inflight first-stream parts and two second-stream parts queued.
 *
 * ckpp_serve_run_plain (the comparison arm) launches one ckpp_bulk_lookup or
 * ckpp_bulk_insert per burst on the burst's own table, in arrival order, as
 * bursts arrive, with one event per group of bursts launched together.
 *
 * Lookup burst b of table t reads keys at pool_keys[t] + 16 * offset[b] and
 * writes values at pool_vals[t] + 8 * offset[b] and flags at pool_found[t] +
 * offset[b] (size[b] keys). Insert burst b uses keys [offset[b], offset[b] +
 * size[b]) of the insert pool, their values, table indices (into the batch's
 * tables, also the stream's table numbers) and status bytes.
 *
 * done_at [n] out: each burst's completion time, seconds since the call's
 * start (its turn's event, on the device clock, offset by the start event).
 * Errors: CKPP_EINVAL (NULL, sizes), any error of the calls it makes (the run
 * stops there; work already queued still runs), CKPP_ECUDA. */
typedef struct ckpp_serve_buffers {
  const uint64_t* pool_keys;   /* host [n_tables]: device address of each table's lookup keys */
  const uint64_t* pool_vals;   /* host [n_tables]: ... of its value outputs */
  const uint64_t* pool_found;  /* host [n_tables]: ... of its found flags */
  uint32_t n_tables;
  uint32_t max_jobs;           /* jobs per batched lookup launch (<= CKPP_BATCH_MAX_JOBS) */
  const ckpp_key* ins_keys;    /* device insert pool (arrival order) */
  const uint32_t* ins_tables;  /* device table index per insert key */
  const uint64_t* ins_vals;    /* device value per insert key */
  uint8_t* ins_status;         /* device status per insert key (out) */
  void* ins_workspace;         /* device workspace for the largest insert call */
  size_t ins_workspace_bytes;
  ckpp_lookup_job* d_jobs;     /* device job records: max_jobs, or ring_slots x max_jobs with overlap */
  ckpp_lookup_job* h_jobs;     /* pinned host memory: ring_slots x max_jobs records */
  uint32_t ring_slots;         /* >= 1 */
  uint32_t max_inflight;       /* ckpp_serve_run: turns queued on the device at most (0: no limit); at the
                                  limit the loop waits for the oldest, and arrivals gather meanwhile */
  ckpp_batch* batch_b;         /* overlap: a second descriptor over the same tables, for the second stream's
                                  lookups (one descriptor's lookup launches must not overlap); else NULL */
} ckpp_serve_buffers;

typedef struct ckpp_serve_stats {
  double wall_s;          /* from the start to the last completion */
  double gpu_busy_s;      /* sum over turns (groups) of the device time of their launches */
  uint64_t turns;         /* turns launched (batched) or launch groups (plain) */
  uint64_t launches;      /* library calls made */
  uint64_t flushes;       /* insert calls (batched) */
  uint64_t held;          /* lookup bursts launched behind a flush (batched) */
  uint64_t admitted;      /* bursts admitted, summed over turns */
  double gpu_busy_b_s;    /* overlap: the same for the second-stream parts (gpu_busy_s then counts the first) */
  uint64_t trailing;      /* overlap: lookup bursts launched behind a flush in flight */
} ckpp_serve_stats;

int ckpp_serve_run(ckpp_planner* planner, ckpp_batch* batch, const ckpp_serve_buffers* buffers,
                   const ckpp_batch_tuning* tuning, ckpp_stream_t stream, double* done_at, ckpp_serve_stats* stats);

/* tables [n_tables]: the handle of each table (the stream's table numbers);
 * the planner only lends the stream and is not advanced. */
int ckpp_serve_run_plain(const ckpp_planner* planner, ckpp_table* const* tables, const ckpp_serve_buffers* buffers,
                         ckpp_stream_t stream, double* done_at, ckpp_serve_stats* stats);

#ifdef __cplusplus
}
#endif

#endif /* CKPP_SERVE_H */
