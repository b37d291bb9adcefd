// The served form's serving loops (include/ckpp_serve.h): host code that runs
// a pre-drawn burst stream in real time and drives the device through the
// library's own entry points, one CUDA stream, no waiting between turns.
//
// Continuous batching: whenever the loop is free it retires the turns whose
// end event has completed (their bursts get their completion time and release
// their footprint), asks the planner for a turn at the current host time, and
// launches it behind the turns already queued. A turn's lookup jobs are staged
// in one slot of a ring of pinned host buffers and copied to the device job
// array ahead of its launches; a slot is reused only after the copy that last
// read it has run (its turn's event). The comparison arm launches one plain
// call per burst as bursts arrive.

#include <chrono>
#include <deque>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "serve_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point t0) {
  return std::chrono::duration<double>(Clock::now() - t0).count();
}

// Events are recycled: a turn takes two (its start and end) and returns them
// when it retires.
struct EventPool {
  std::vector<cudaEvent_t> free, all;
  cudaError_t get(cudaEvent_t& e) {
    if (!free.empty()) {
      e = free.back();
      free.pop_back();
      return cudaSuccess;
    }
    const cudaError_t r = cudaEventCreate(&e);
    if (r == cudaSuccess) all.push_back(e);
    return r;
  }
  void put(cudaEvent_t e) { free.push_back(e); }
  ~EventPool() {
    for (cudaEvent_t e : all) cudaEventDestroy(e);
  }
};

struct InFlight {
  cudaEvent_t start, end;
  std::vector<int64_t> bursts;  // the bursts the turn completes
  int64_t nbytes;
  int ring_slot;                // the staging slot its copy read, or -1
};

// Device time of ev after the start event, in seconds.
cudaError_t event_seconds(cudaEvent_t start, cudaEvent_t ev, double& s) {
  float ms = 0.f;
  const cudaError_t r = cudaEventElapsedTime(&ms, start, ev);
  s = ms * 1e-3;
  return r;
}

bool buffers_ok(const ckpp_serve_buffers* b, const ckpp_planner* p) {
  if (!b || !b->pool_keys || !b->pool_vals || !b->pool_found || b->ring_slots < 1 || b->max_jobs < 1 ||
      b->max_jobs > CKPP_BATCH_MAX_JOBS || !b->d_jobs || !b->h_jobs)
    return false;
  for (int64_t i = 0; i < p->n; ++i)
    if (p->table[i] >= b->n_tables) return false;
  return true;
}

}  // namespace

namespace {
int serve_run_overlap(ckpp_planner* p, ckpp_batch* batch, const ckpp_serve_buffers* buf,
                      const ckpp_batch_tuning* tuning, cudaStream_t s, double* done_at, ckpp_serve_stats* stats);
}  // namespace

extern "C" int ckpp_serve_run(ckpp_planner* p, ckpp_batch* batch, const ckpp_serve_buffers* buf,
                              const ckpp_batch_tuning* tuning, ckpp_stream_t stream, double* done_at,
                              ckpp_serve_stats* stats) {
  if (!p || !batch || !done_at || !stats || !buffers_ok(buf, p) || p->cfg.max_jobs > buf->max_jobs) return CKPP_EINVAL;
  const int64_t n = p->n;
  if (n > 0 && (!buf->ins_keys || !buf->ins_tables || !buf->ins_vals || !buf->ins_status)) {
    for (int64_t b = 0; b < n; ++b)
      if (p->insert[b]) return CKPP_EINVAL;
  }
  if (p->cfg.overlap) {
    if (!buf->batch_b || buf->batch_b == batch) return CKPP_EINVAL;
    return serve_run_overlap(p, batch, buf, tuning, reinterpret_cast<cudaStream_t>(stream), done_at, stats);
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  *stats = ckpp_serve_stats{};
  std::vector<int64_t> lookups(n > 0 ? n : 1), inserts(n > 0 ? n : 1), after(n > 0 ? n : 1), jobs_idx;
  std::vector<cudaEvent_t> ring_event(buf->ring_slots, nullptr);  // the end event of the slot's last reader
  std::deque<InFlight> flight;
  EventPool events;
  cudaEvent_t e0;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return CKPP_ECUDA;
  const Clock::time_point t0 = Clock::now();
  if (cudaEventRecord(e0, s) != cudaSuccess) {
    cudaEventDestroy(e0);
    return CKPP_ECUDA;
  }
  int rc = CKPP_OK;
  uint32_t slot = 0;
  double last_done = 0.0;
  auto retire = [&](bool block) -> int {
    while (!flight.empty()) {
      InFlight& f = flight.front();
      cudaError_t q = block ? cudaEventSynchronize(f.end) : cudaEventQuery(f.end);
      if (q == cudaErrorNotReady) return CKPP_OK;
      if (q != cudaSuccess) return CKPP_ECUDA;
      double t_end = 0, busy = 0;
      if (event_seconds(e0, f.end, t_end) != cudaSuccess || event_seconds(f.start, f.end, busy) != cudaSuccess)
        return CKPP_ECUDA;
      for (int64_t b : f.bursts) done_at[b] = t_end;
      last_done = t_end > last_done ? t_end : last_done;
      stats->gpu_busy_s += busy;
      if (ckpp_plan_complete(p, f.nbytes) != CKPP_OK) return CKPP_EINVAL;
      if (f.ring_slot >= 0 && ring_event[f.ring_slot] == f.end) ring_event[f.ring_slot] = nullptr;
      events.put(f.start);
      events.put(f.end);
      flight.pop_front();
      block = false;
    }
    return CKPP_OK;
  };
  for (;;) {
    int fin = 0;
    ckpp_plan_state(p, nullptr, nullptr, &fin);
    if (fin && flight.empty()) break;
    if ((rc = retire(false)) != CKPP_OK) break;
    if (buf->max_inflight && flight.size() >= buf->max_inflight) {  // pace the turns to the device
      if ((rc = retire(true)) != CKPP_OK) break;
      continue;
    }
    const double now = seconds_since(t0);
    ckpp_turn turn;
    if ((rc = ckpp_plan_next(p, now, flight.empty() ? 0 : 1, &turn, lookups.data(), nullptr, inserts.data(),
                             after.data(), n)) != CKPP_OK)
      break;
    if (turn.action == CKPP_PLAN_IDLE) {
      if (flight.empty()) {
        const double wait = turn.wake - now;
        if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(wait < 50e-6 ? wait : 50e-6));
      }
      continue;
    }
    if (turn.action == CKPP_PLAN_BLOCK) {
      if ((rc = retire(true)) != CKPP_OK) break;
      continue;
    }
    if (turn.action == CKPP_PLAN_NONE) continue;
    // the turn's host work first, so that its launches go out back to back
    const int64_t nj = turn.n_lookups + turn.n_after;
    int used_slot = -1;
    if (nj) {
      if (ring_event[slot] && cudaEventSynchronize(ring_event[slot]) != cudaSuccess) {
        rc = CKPP_ECUDA;
        break;
      }
      jobs_idx.assign(lookups.begin(), lookups.begin() + turn.n_lookups);
      jobs_idx.insert(jobs_idx.end(), after.begin(), after.begin() + turn.n_after);
      ckpp_lookup_job* h = buf->h_jobs + (size_t)slot * buf->max_jobs;
      ckpp_serve_stage_jobs(jobs_idx.data(), nj, p->table, p->offset, p->size, buf->pool_keys, buf->pool_vals,
                            buf->pool_found, h);
      if (cudaMemcpyAsync(buf->d_jobs, h, (size_t)nj * sizeof(ckpp_lookup_job), cudaMemcpyHostToDevice, s) !=
          cudaSuccess) {
        rc = CKPP_ECUDA;
        break;
      }
      used_slot = (int)slot;
    }
    InFlight f;
    if (events.get(f.start) != cudaSuccess || events.get(f.end) != cudaSuccess ||
        cudaEventRecord(f.start, s) != cudaSuccess) {
      rc = CKPP_ECUDA;
      break;
    }
    if (turn.n_lookups) {  // 1. lookups whose table has no waiting insert
      if ((rc = ckpp_batch_lookup(batch, buf->d_jobs, (uint32_t)turn.n_lookups, nullptr, 0, tuning, stream)))
        break;
      ++stats->launches;
    }
    if (turn.n_inserts) {  // 2. the waiting inserts, one contiguous range of the insert pool
      const int64_t first = turn.insert_first;
      if ((rc = ckpp_batch_insert(batch, buf->ins_keys + first, buf->ins_tables + first, buf->ins_vals + first,
                                  (uint64_t)turn.insert_keys, 0, 0, buf->ins_status + first, buf->ins_workspace,
                                  buf->ins_workspace_bytes, stream)))
        break;
      ++stats->launches;
      ++stats->flushes;
    }
    if (turn.n_after) {  // 3. lookups held behind those inserts
      if ((rc = ckpp_batch_lookup(batch, buf->d_jobs + turn.n_lookups, (uint32_t)turn.n_after, nullptr, 0, tuning,
                                  stream)))
        break;
      ++stats->launches;
      stats->held += (uint64_t)turn.n_after;
    }
    if (cudaEventRecord(f.end, s) != cudaSuccess) {
      rc = CKPP_ECUDA;
      break;
    }
    f.bursts.reserve((size_t)(turn.n_lookups + turn.n_inserts + turn.n_after));
    f.bursts.insert(f.bursts.end(), lookups.begin(), lookups.begin() + turn.n_lookups);
    f.bursts.insert(f.bursts.end(), inserts.begin(), inserts.begin() + turn.n_inserts);
    f.bursts.insert(f.bursts.end(), after.begin(), after.begin() + turn.n_after);
    f.nbytes = turn.nbytes;
    f.ring_slot = used_slot;
    if (used_slot >= 0) {
      ring_event[used_slot] = f.end;
      slot = (slot + 1) % buf->ring_slots;
    }
    flight.push_back(std::move(f));
    ++stats->turns;
    stats->admitted += (uint64_t)(turn.admitted_hi - turn.admitted_lo);
  }
  if (rc != CKPP_OK) {
    cudaStreamSynchronize(s);  // leave nothing queued that reads the staging buffers
  } else {
    rc = retire(true);
  }
  stats->wall_s = last_done;
  cudaEventDestroy(e0);
  return rc;
}

extern "C" int ckpp_serve_run_plain(const ckpp_planner* p, ckpp_table* const* tables,
                                    const ckpp_serve_buffers* buf, ckpp_stream_t stream, double* done_at,
                                    ckpp_serve_stats* stats) {
  if (!p || !tables || !done_at || !stats || !buffers_ok(buf, p)) return CKPP_EINVAL;
  const int64_t n = p->n;
  for (uint32_t t = 0; t < buf->n_tables; ++t)
    if (!tables[t]) return CKPP_EINVAL;
  for (int64_t b = 0; b < n; ++b)
    if (p->insert[b] && (!buf->ins_keys || !buf->ins_vals || !buf->ins_status)) return CKPP_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  *stats = ckpp_serve_stats{};
  std::deque<InFlight> flight;
  EventPool events;
  cudaEvent_t e0;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return CKPP_ECUDA;
  const Clock::time_point t0 = Clock::now();
  if (cudaEventRecord(e0, s) != cudaSuccess) {
    cudaEventDestroy(e0);
    return CKPP_ECUDA;
  }
  int rc = CKPP_OK;
  double last_done = 0.0;
  int64_t nxt = 0;
  auto retire = [&](bool block) -> int {
    while (!flight.empty()) {
      InFlight& f = flight.front();
      cudaError_t q = block ? cudaEventSynchronize(f.end) : cudaEventQuery(f.end);
      if (q == cudaErrorNotReady) return CKPP_OK;
      if (q != cudaSuccess) return CKPP_ECUDA;
      double t_end = 0, busy = 0;
      if (event_seconds(e0, f.end, t_end) != cudaSuccess || event_seconds(f.start, f.end, busy) != cudaSuccess)
        return CKPP_ECUDA;
      for (int64_t b : f.bursts) done_at[b] = t_end;
      last_done = t_end > last_done ? t_end : last_done;
      stats->gpu_busy_s += busy;
      events.put(f.start);
      events.put(f.end);
      flight.pop_front();
      block = false;
    }
    return CKPP_OK;
  };
  while (nxt < n || !flight.empty()) {
    if ((rc = retire(false)) != CKPP_OK) break;
    const double now = seconds_since(t0);
    if (nxt < n && p->arrival[nxt] <= now) {
      InFlight f;
      if (events.get(f.start) != cudaSuccess || events.get(f.end) != cudaSuccess ||
          cudaEventRecord(f.start, s) != cudaSuccess) {
        rc = CKPP_ECUDA;
        break;
      }
      const int64_t hi = std::upper_bound(p->arrival + nxt, p->arrival + n, now) - p->arrival;
      for (int64_t b = nxt; b < hi && rc == CKPP_OK; ++b) {
        const uint32_t t = p->table[b];
        const int64_t off = p->offset[b];
        if (p->insert[b]) {
          rc = ckpp_bulk_insert(tables[t], buf->ins_keys + off, buf->ins_vals + off, p->size[b], 0, 0,
                                buf->ins_status + off, buf->ins_workspace, buf->ins_workspace_bytes, stream);
        } else {
          rc = ckpp_bulk_lookup(tables[t], reinterpret_cast<const ckpp_key*>(buf->pool_keys[t] + 16 * (uint64_t)off),
                                p->size[b], reinterpret_cast<uint64_t*>(buf->pool_vals[t] + 8 * (uint64_t)off),
                                reinterpret_cast<uint8_t*>(buf->pool_found[t] + (uint64_t)off), 0, 0, stream);
        }
        ++stats->launches;
      }
      if (rc != CKPP_OK) break;
      if (cudaEventRecord(f.end, s) != cudaSuccess) {
        rc = CKPP_ECUDA;
        break;
      }
      for (int64_t b = nxt; b < hi; ++b) f.bursts.push_back(b);
      f.nbytes = 0;
      f.ring_slot = -1;
      flight.push_back(std::move(f));
      ++stats->turns;
      stats->admitted += (uint64_t)(hi - nxt);
      nxt = hi;
    } else if (flight.empty() && nxt < n) {
      const double wait = p->arrival[nxt] - now;
      if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(wait < 50e-6 ? wait : 50e-6));
    }
  }
  if (rc != CKPP_OK) {
    cudaStreamSynchronize(s);
  } else {
    rc = retire(true);
  }
  stats->wall_s = last_done;
  cudaEventDestroy(e0);
  return rc;
}

namespace {

// One stream's part of a turn, in flight.
struct Part {
  cudaEvent_t start, end;
  std::vector<int64_t> bursts;
  int64_t nbytes;
  bool flushed;   // second-stream part carrying a flush
  int ring_slot;
};

// Continuous batching with the flushes on a second stream (the planner's
// overlap mode): a turn's free lookups go to the caller's stream; its trailing
// lookups, flush and held lookups to the second stream, after an event wait on
// the first (so a flush follows every lookup launched before it). The second
// stream's lookups use their own batch descriptor (buf->batch_b): a
// descriptor's work counters serve one launch at a time. Each turn
// stages its jobs in its own ring slot of host and device job records
// (ring_slots x max_jobs each), reused only after both parts that read it ran.
int serve_run_overlap(ckpp_planner* p, ckpp_batch* batch, const ckpp_serve_buffers* buf,
                      const ckpp_batch_tuning* tuning, cudaStream_t s, double* done_at, ckpp_serve_stats* stats) {
  const int64_t n = p->n;
  *stats = ckpp_serve_stats{};
  std::vector<int64_t> lookups(n > 0 ? n : 1), trailing(n > 0 ? n : 1), inserts(n > 0 ? n : 1),
      after(n > 0 ? n : 1), jobs_idx;
  std::vector<cudaEvent_t> ring_a(buf->ring_slots, nullptr), ring_b(buf->ring_slots, nullptr);
  std::deque<Part> flight_a, flight_b;
  EventPool events;
  cudaStream_t sb;
  if (cudaStreamCreateWithFlags(&sb, cudaStreamNonBlocking) != cudaSuccess) return CKPP_ECUDA;
  cudaEvent_t e0;
  if (cudaEventCreate(&e0) != cudaSuccess) {
    cudaStreamDestroy(sb);
    return CKPP_ECUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaStreamDestroy(sb);
    return CKPP_ECUDA;
  }
  const Clock::time_point t0 = Clock::now();
  int rc = cudaEventRecord(e0, s) == cudaSuccess ? CKPP_OK : CKPP_ECUDA;
  uint32_t slot = 0;
  double last_done = 0.0;
  const ckpp_stream_t ha = reinterpret_cast<ckpp_stream_t>(s), hb = reinterpret_cast<ckpp_stream_t>(sb);
  // retire the completed parts of one stream (block: wait for its oldest part first)
  auto retire = [&](std::deque<Part>& q, std::vector<cudaEvent_t>& ring, bool second, bool block) -> int {
    while (!q.empty()) {
      Part& f = q.front();
      const cudaError_t st = block ? cudaEventSynchronize(f.end) : cudaEventQuery(f.end);
      if (st == cudaErrorNotReady) return CKPP_OK;
      if (st != cudaSuccess) return CKPP_ECUDA;
      double t_end = 0, busy = 0;
      if (event_seconds(e0, f.end, t_end) != cudaSuccess || event_seconds(f.start, f.end, busy) != cudaSuccess)
        return CKPP_ECUDA;
      for (int64_t b : f.bursts) done_at[b] = t_end;
      last_done = t_end > last_done ? t_end : last_done;
      if (second) {
        stats->gpu_busy_b_s += busy;
        if (ckpp_plan_complete_b(p, f.nbytes, f.flushed ? 1 : 0) != CKPP_OK) return CKPP_EINVAL;
      } else {
        stats->gpu_busy_s += busy;
        if (ckpp_plan_complete(p, f.nbytes) != CKPP_OK) return CKPP_EINVAL;
      }
      if (f.ring_slot >= 0 && ring[f.ring_slot] == f.end) ring[f.ring_slot] = nullptr;
      events.put(f.start);
      events.put(f.end);
      q.pop_front();
      block = false;
    }
    return CKPP_OK;
  };
  while (rc == CKPP_OK) {
    int fin = 0;
    ckpp_plan_state(p, nullptr, nullptr, &fin);
    if (fin && flight_a.empty() && flight_b.empty()) break;
    if ((rc = retire(flight_a, ring_a, false, false)) != CKPP_OK) break;
    if ((rc = retire(flight_b, ring_b, true, false)) != CKPP_OK) break;
    // pace the first stream as the one-stream loop does, and keep at most two parts on the second
    if (buf->max_inflight && flight_a.size() >= buf->max_inflight) {
      rc = retire(flight_a, ring_a, false, true);
      continue;
    }
    if (flight_b.size() >= 2) {
      rc = retire(flight_b, ring_b, true, true);
      continue;
    }
    const double now = seconds_since(t0);
    ckpp_turn turn;
    const int outstanding = (flight_a.empty() && flight_b.empty()) ? 0 : 1;
    if ((rc = ckpp_plan_next(p, now, outstanding, &turn, lookups.data(), trailing.data(), inserts.data(),
                             after.data(), n)) != CKPP_OK)
      break;
    if (turn.action == CKPP_PLAN_IDLE) {
      if (!outstanding) {
        const double wait = turn.wake - now;
        if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(wait < 50e-6 ? wait : 50e-6));
      }
      continue;
    }
    if (turn.action == CKPP_PLAN_BLOCK) {  // wait for the older of the two streams' oldest parts
      if (!flight_a.empty()) {
        rc = retire(flight_a, ring_a, false, true);
      } else {
        rc = retire(flight_b, ring_b, true, true);
      }
      continue;
    }
    if (turn.action == CKPP_PLAN_NONE) continue;
    const int64_t nj = turn.n_lookups + turn.n_trailing + turn.n_after;
    const bool has_b = turn.n_trailing || turn.n_inserts || turn.n_after;
    ckpp_lookup_job* d = buf->d_jobs + (size_t)slot * buf->max_jobs;
    int used_slot = -1;
    if (nj) {
      for (cudaEvent_t e : {ring_a[slot], ring_b[slot]})
        if (e && cudaEventSynchronize(e) != cudaSuccess) rc = CKPP_ECUDA;
      if (rc != CKPP_OK) break;
      jobs_idx.assign(lookups.begin(), lookups.begin() + turn.n_lookups);
      jobs_idx.insert(jobs_idx.end(), trailing.begin(), trailing.begin() + turn.n_trailing);
      jobs_idx.insert(jobs_idx.end(), after.begin(), after.begin() + turn.n_after);
      ckpp_lookup_job* h = buf->h_jobs + (size_t)slot * buf->max_jobs;
      ckpp_serve_stage_jobs(jobs_idx.data(), nj, p->table, p->offset, p->size, buf->pool_keys, buf->pool_vals,
                            buf->pool_found, h);
      if (cudaMemcpyAsync(d, h, (size_t)nj * sizeof(ckpp_lookup_job), cudaMemcpyHostToDevice, s) != cudaSuccess) {
        rc = CKPP_ECUDA;
        break;
      }
      used_slot = (int)slot;
    }
    Part a;
    if (events.get(a.start) != cudaSuccess || events.get(a.end) != cudaSuccess ||
        cudaEventRecord(a.start, s) != cudaSuccess) {
      rc = CKPP_ECUDA;
      break;
    }
    if (turn.n_lookups) {  // free lookups on the first stream
      if ((rc = ckpp_batch_lookup(batch, d, (uint32_t)turn.n_lookups, nullptr, 0, tuning, ha))) break;
      ++stats->launches;
    }
    if (cudaEventRecord(a.end, s) != cudaSuccess) {
      rc = CKPP_ECUDA;
      break;
    }
    if (has_b) {
      Part b;
      if (cudaStreamWaitEvent(sb, a.end, 0) != cudaSuccess || events.get(b.start) != cudaSuccess ||
          events.get(b.end) != cudaSuccess || cudaEventRecord(b.start, sb) != cudaSuccess) {
        rc = CKPP_ECUDA;
        break;
      }
      if (turn.n_trailing) {  // behind the flushes in flight
        if ((rc = ckpp_batch_lookup(buf->batch_b, d + turn.n_lookups, (uint32_t)turn.n_trailing, nullptr, 0, tuning,
                                    hb)))
          break;
        ++stats->launches;
        stats->trailing += (uint64_t)turn.n_trailing;
      }
      if (turn.n_inserts) {
        const int64_t first = turn.insert_first;
        if ((rc = ckpp_batch_insert(batch, buf->ins_keys + first, buf->ins_tables + first, buf->ins_vals + first,
                                    (uint64_t)turn.insert_keys, 0, 0, buf->ins_status + first, buf->ins_workspace,
                                    buf->ins_workspace_bytes, hb)))
          break;
        ++stats->launches;
        ++stats->flushes;
      }
      if (turn.n_after) {
        if ((rc = ckpp_batch_lookup(buf->batch_b, d + turn.n_lookups + turn.n_trailing, (uint32_t)turn.n_after,
                                    nullptr, 0, tuning, hb)))
          break;
        ++stats->launches;
        stats->held += (uint64_t)turn.n_after;
      }
      if (cudaEventRecord(b.end, sb) != cudaSuccess) {
        rc = CKPP_ECUDA;
        break;
      }
      b.bursts.insert(b.bursts.end(), trailing.begin(), trailing.begin() + turn.n_trailing);
      b.bursts.insert(b.bursts.end(), inserts.begin(), inserts.begin() + turn.n_inserts);
      b.bursts.insert(b.bursts.end(), after.begin(), after.begin() + turn.n_after);
      b.nbytes = turn.nbytes_b;
      b.flushed = turn.n_inserts > 0;
      b.ring_slot = used_slot;
      if (used_slot >= 0) ring_b[used_slot] = b.end;
      flight_b.push_back(std::move(b));
    }
    a.bursts.assign(lookups.begin(), lookups.begin() + turn.n_lookups);
    a.nbytes = turn.nbytes;
    a.flushed = false;
    a.ring_slot = used_slot;
    if (used_slot >= 0) {
      ring_a[used_slot] = a.end;
      slot = (slot + 1) % buf->ring_slots;
    }
    flight_a.push_back(std::move(a));
    ++stats->turns;
    stats->admitted += (uint64_t)(turn.admitted_hi - turn.admitted_lo);
  }
  if (rc != CKPP_OK) {
    cudaStreamSynchronize(s);
    cudaStreamSynchronize(sb);
  } else {
    rc = retire(flight_a, ring_a, false, true);
    if (rc == CKPP_OK) rc = retire(flight_b, ring_b, true, true);
  }
  stats->wall_s = last_done;
  cudaEventDestroy(e0);
  cudaStreamDestroy(sb);
  return rc;
}

}  // namespace
