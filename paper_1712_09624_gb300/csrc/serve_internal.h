// Internal state of the served form's turn planner (include/ckpp_serve.h),
// shared by the planner (serve_plan.cpp) and the native serving loops
// (serve_run.cu), which read the stream arrays it borrows.
#pragma once

#include <algorithm>
#include <cstdint>
#include <deque>
#include <vector>

#include "../../include/ckpp.h"
#include "../../include/ckpp_serve.h"

namespace ckpp_serve {

constexpr uint32_t kMaxTables = 1u << 20;

}  // namespace ckpp_serve

struct ckpp_planner {
  const double* arrival;
  const uint32_t* table;
  const uint32_t* size;
  const uint8_t* insert;
  const int64_t* offset;
  int64_t n;
  ckpp_plan_config cfg;
  int64_t nxt = 0;                 // first burst not yet admitted
  std::vector<int64_t> pending;    // admitted insert bursts not yet launched
  int64_t pending_keys = 0;
  std::vector<int64_t> held;       // admitted lookups waiting for the flush
  std::vector<uint8_t> pend_mask;  // per table: an insert waits
  std::vector<uint8_t> held_mask;  // per table: a lookup is held
  std::vector<int64_t> lookups;    // scratch: this turn's free lookups
  std::vector<int64_t> trailing;   // scratch (overlap): this turn's lookups behind a flush in flight
  std::vector<uint32_t> flight_cnt;              // overlap, per table: flushes in flight holding its inserts
  std::deque<std::vector<uint32_t>> flushes;     // overlap: the tables of each flush in flight, in launch order
  int64_t flight_bytes = 0;        // footprint admitted and not yet completed

  int64_t foot(int64_t b) const { return int64_t(size[b]) * int64_t(cfg.bytes_per_key); }

  bool flush_due(double now) const {
    if (pending.empty()) return false;
    return uint64_t(pending_keys) >= cfg.insert_flush_keys || nxt >= n ||
           now - arrival[pending.front()] >= cfg.insert_flush_s ||
           (!held.empty() && now - arrival[held.front()] >= cfg.lookup_hold_s);
  }

  double wake(double now) const {
    double w = nxt < n ? arrival[nxt] : now;
    if (!pending.empty()) w = std::min(w, arrival[pending.front()] + cfg.insert_flush_s);
    if (!held.empty()) w = std::min(w, arrival[held.front()] + cfg.lookup_hold_s);
    return w;
  }
};

