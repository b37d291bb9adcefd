// Turn planner and job staging of the served form: host code only (no CUDA).
//
// The rules are the ones include/ckpp_serve.h states. The planner walks the
// admitted bursts one at a time with two per-table flags: a table has a
// waiting insert (its lookups are held until the flush) and a table has a held
// lookup (its next insert must wait for the flush). Both flags are cleared at
// each flush by walking the flushed bursts, so a turn costs time in the
// bursts it touches, not in the number of tables.

#include <cstring>
#include <new>

#include "serve_internal.h"

using ckpp_serve::kMaxTables;

extern "C" int ckpp_plan_create(const double* arrival, const uint32_t* table, const uint32_t* size,
                                const uint8_t* insert, const int64_t* offset, int64_t n, const ckpp_plan_config* cfg,
                                ckpp_planner** out) {
  if (!out || !cfg || n < 0 || (n > 0 && (!arrival || !table || !size || !insert || !offset))) return CKPP_EINVAL;
  if (cfg->max_jobs < 1 || cfg->bytes_per_key < 1 || !(cfg->insert_flush_s >= 0) || !(cfg->lookup_hold_s >= 0) ||
      cfg->overlap > 1)
    return CKPP_EINVAL;
  uint32_t n_tables = 1;
  for (int64_t b = 0; b < n; ++b) {
    if (table[b] >= kMaxTables) return CKPP_EINVAL;
    if (b > 0 && !(arrival[b] >= arrival[b - 1])) return CKPP_EINVAL;
    n_tables = std::max(n_tables, table[b] + 1);
  }
  ckpp_planner* p = new (std::nothrow) ckpp_planner();
  if (!p) return CKPP_EINVAL;
  p->arrival = arrival;
  p->table = table;
  p->size = size;
  p->insert = insert;
  p->offset = offset;
  p->n = n;
  p->cfg = *cfg;
  try {
    p->pend_mask.assign(n_tables, 0);
    p->held_mask.assign(n_tables, 0);
    p->flight_cnt.assign(n_tables, 0);
  } catch (...) {
    delete p;
    return CKPP_EINVAL;
  }
  *out = p;
  return CKPP_OK;
}

extern "C" int ckpp_plan_destroy(ckpp_planner* p) {
  delete p;
  return CKPP_OK;
}

extern "C" int ckpp_plan_next(ckpp_planner* p, double now, int outstanding, ckpp_turn* turn, int64_t* lookups,
                              int64_t* trailing, int64_t* inserts, int64_t* after, int64_t cap) {
  if (!p || !turn || !lookups || !inserts || !after || cap < 0 || (p->cfg.overlap && !trailing)) return CKPP_EINVAL;
  std::memset(turn, 0, sizeof(*turn));
  const int64_t n = p->n;
  const bool arrived = p->nxt < n && p->arrival[p->nxt] <= now;
  bool flush = p->flush_due(now);
  if (!arrived && !flush) {
    turn->action = CKPP_PLAN_IDLE;
    turn->wake = p->wake(now);
    turn->admitted_lo = turn->admitted_hi = p->nxt;
    return CKPP_OK;
  }
  // the turn returns at most the waiting bursts and the new arrivals: check the caller's room first
  const int64_t lo = p->nxt;
  const int64_t hi = arrived ? std::upper_bound(p->arrival + lo, p->arrival + n, now) - p->arrival : lo;
  if (int64_t(p->pending.size() + p->held.size()) + (hi - lo) > cap) return CKPP_EINVAL;
  p->lookups.clear();
  p->trailing.clear();
  int64_t stop = lo;
  if (arrived) {
    const int64_t room = int64_t(p->cfg.footprint_bytes) - p->flight_bytes;
    int64_t fit = 0, acc = 0;
    while (lo + fit < hi && acc + p->foot(lo + fit) <= room) acc += p->foot(lo + fit++);
    if (fit == 0) {
      if (!p->pending.empty()) {
        flush = true;  // waiting inserts hold the budget: send them
      } else if (outstanding) {
        turn->action = CKPP_PLAN_BLOCK;
        turn->admitted_lo = turn->admitted_hi = lo;
        return CKPP_OK;
      } else {
        fit = 1;  // a burst larger than the budget goes alone
      }
    }
    for (int64_t b = lo; b < lo + fit; ++b) {
      const uint32_t t = p->table[b];
      if (p->insert[b]) {
        if (p->held_mask[t]) {
          flush = true;  // a held lookup of t must not see this insert: flush first
          break;
        }
        p->pending.push_back(b);
        p->pending_keys += p->size[b];
        p->pend_mask[t] = 1;
      } else {
        if (p->lookups.size() + p->trailing.size() + p->held.size() >= p->cfg.max_jobs) {
          flush = true;  // the job array is full (flushes only if inserts wait)
          break;
        }
        if (p->pend_mask[t]) {
          p->held.push_back(b);
          p->held_mask[t] = 1;
        } else if (p->flight_cnt[t]) {
          p->trailing.push_back(b);  // behind the flush in flight on the second stream
        } else {
          p->lookups.push_back(b);
        }
      }
      stop = b + 1;
    }
    for (int64_t b = lo; b < stop; ++b) p->flight_bytes += p->foot(b);
    p->nxt = stop;
  }
  turn->admitted_lo = lo;
  turn->admitted_hi = stop;
  flush = !p->pending.empty() && (flush || p->flush_due(now));
  if (p->lookups.empty() && p->trailing.empty() && !flush) {
    turn->action = CKPP_PLAN_NONE;
    return CKPP_OK;
  }
  turn->action = CKPP_PLAN_LAUNCH;
  int64_t nbytes = 0, nbytes_b = 0;
  turn->n_lookups = int64_t(p->lookups.size());
  for (size_t i = 0; i < p->lookups.size(); ++i) {
    lookups[i] = p->lookups[i];
    nbytes += p->foot(p->lookups[i]);
  }
  turn->n_trailing = int64_t(p->trailing.size());
  for (size_t i = 0; i < p->trailing.size(); ++i) {
    trailing[i] = p->trailing[i];
    nbytes_b += p->foot(p->trailing[i]);
  }
  if (flush) {
    turn->n_inserts = int64_t(p->pending.size());
    turn->insert_first = p->offset[p->pending.front()];
    turn->insert_keys = p->pending_keys;
    std::vector<uint32_t> tables;  // overlap: the flush's tables, each once
    for (size_t i = 0; i < p->pending.size(); ++i) {
      const int64_t b = p->pending[i];
      inserts[i] = b;
      nbytes_b += p->foot(b);
      if (p->cfg.overlap && p->pend_mask[p->table[b]]) {
        tables.push_back(p->table[b]);
        ++p->flight_cnt[p->table[b]];
      }
      p->pend_mask[p->table[b]] = 0;
    }
    if (p->cfg.overlap) p->flushes.push_back(std::move(tables));
    turn->n_after = int64_t(p->held.size());
    for (size_t i = 0; i < p->held.size(); ++i) {
      const int64_t b = p->held[i];
      after[i] = b;
      nbytes_b += p->foot(b);
      p->held_mask[p->table[b]] = 0;
    }
    p->pending.clear();
    p->pending_keys = 0;
    p->held.clear();
  }
  if (p->cfg.overlap) {
    turn->nbytes = nbytes;
    turn->nbytes_b = nbytes_b;
  } else {
    turn->nbytes = nbytes + nbytes_b;
  }
  return CKPP_OK;
}

extern "C" int ckpp_plan_complete_b(ckpp_planner* p, int64_t nbytes_b, int flushed) {
  if (!p || !p->cfg.overlap || nbytes_b < 0 || nbytes_b > p->flight_bytes || (flushed && p->flushes.empty()))
    return CKPP_EINVAL;
  p->flight_bytes -= nbytes_b;
  if (flushed) {
    for (uint32_t t : p->flushes.front()) --p->flight_cnt[t];
    p->flushes.pop_front();
  }
  return CKPP_OK;
}

extern "C" int ckpp_plan_complete(ckpp_planner* p, int64_t nbytes) {
  if (!p || nbytes < 0 || nbytes > p->flight_bytes) return CKPP_EINVAL;
  p->flight_bytes -= nbytes;
  return CKPP_OK;
}

extern "C" int ckpp_plan_state(const ckpp_planner* p, int64_t* pending_keys, int64_t* flight_bytes, int* finished) {
  if (!p) return CKPP_EINVAL;
  if (pending_keys) *pending_keys = p->pending_keys;
  if (flight_bytes) *flight_bytes = p->flight_bytes;
  if (finished) *finished = p->nxt >= p->n && p->pending.empty() && p->held.empty();
  return CKPP_OK;
}

extern "C" int ckpp_serve_stage_jobs(const int64_t* bursts, int64_t n_bursts, const uint32_t* table,
                                     const int64_t* offset, const uint32_t* size, const uint64_t* pool_keys,
                                     const uint64_t* pool_vals, const uint64_t* pool_found, void* jobs) {
  if (n_bursts < 0) return CKPP_EINVAL;
  if (n_bursts == 0) return CKPP_OK;
  if (!bursts || !table || !offset || !size || !pool_keys || !pool_vals || !pool_found || !jobs) return CKPP_EINVAL;
  ckpp_lookup_job* out = static_cast<ckpp_lookup_job*>(jobs);
  for (int64_t i = 0; i < n_bursts; ++i) {
    const int64_t b = bursts[i];
    const uint32_t t = table[b];
    const uint64_t off = uint64_t(offset[b]);
    out[i].keys = reinterpret_cast<const ckpp_key*>(pool_keys[t] + 16 * off);
    out[i].out_vals = reinterpret_cast<uint64_t*>(pool_vals[t] + 8 * off);
    out[i].out_found = reinterpret_cast<uint8_t*>(pool_found[t] + off);
    out[i].n = size[b];
    out[i].table = t;
  }
  return CKPP_OK;
}
