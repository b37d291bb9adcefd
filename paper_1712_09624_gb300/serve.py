"""Served form: a continuous-batching request loop over device-resident tables.

Packet bursts arrive from many ports (``serve_policy.draw_stream``). The loop
runs in real time on the host:

* it retires finished launches (CUDA event queries) and frees their staging
  footprint;
* it asks the turn planner (``serve_policy.TurnPlanner``: admission within an
  HBM footprint budget, write coalescing) what to launch;
* it launches that without waiting for the previous launch, all on one
  stream, in the turn's order: the lookups whose table has no waiting insert
  as one persistent ``ckpp_batch_lookup`` (one job per burst); when the
  planner flushes them, the waiting inserts as one multi-table
  ``ckpp_batch_insert`` (an insert call has a fixed cost of several dependent
  kernels, so coalescing writes keeps that cost from every turn); then the
  lookups that were held behind those inserts as a second batched lookup. The
  next turn is queued while the current one runs.

Each table applies its lookups and inserts in arrival order (the planner's
rule), so every burst gets the result it gets when every burst runs alone in
arrival order. Lookups read flows of the warm fill, unknown flows, and (a
``raw_fraction`` of their keys) flows inserted by earlier insert bursts of
the same table during the run; the tests compare every result with that
sequential answer. Per-burst latency is completion time (the launch's CUDA
event, mapped to host time) minus arrival time.

The comparison arm serves the same arrival stream with one plain launch per
burst (``ckpp_bulk_lookup`` / ``ckpp_bulk_insert``) as bursts arrive.
"""

from __future__ import annotations

import ctypes
import time
from collections import deque

import numpy as np
import torch

from . import _ckpp as K
from . import workload_gpu as WG
from .batched import BatchedLookup
from .serve_policy import ServeConfig, Stream, TurnPlanner, draw_stream  # noqa: F401 (re-exported)
from .table import FlowTable


def percentiles(lat: np.ndarray) -> dict | None:
    if lat.size == 0:
        return None
    return {"p50": round(float(np.percentile(lat, 50)), 1), "p99": round(float(np.percentile(lat, 99)), 1),
            "p99_9": round(float(np.percentile(lat, 99.9)), 1), "max": round(float(lat.max()), 1)}


class Service:
    """Tables, request pools and output buffers of one served run."""

    def __init__(self, cfg: ServeConfig, device=None):
        self.cfg = cfg
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        dev = self.device
        self.stream = draw_stream(cfg)
        st = self.stream
        nb_table = max(2, cfg.total_slots // (8 * cfg.n_tables))
        self.warm = int(cfg.warm_lf * nb_table * 8)
        ws = torch.empty(K.ckpp_workspace_bytes(self.warm), dtype=torch.uint8, device=dev)
        cuda = torch.cuda.current_stream(dev)
        self.tables = []
        for t in range(cfg.n_tables):
            tb = FlowTable(nb_table, seed=cfg.seed * 1000 + t, device=dev)
            k, v = WG.fill_keys(cfg.seed * 1000 + t, 0, self.warm, dev)
            s = torch.empty(self.warm, dtype=torch.uint8, device=dev)
            K.ckpp_bulk_insert(tb.handle, k, v, s, ws, 0, 0, cuda)
            self.tables.append(tb)
        del ws
        # one insert pool for all tables, arrival order: new flows never in any table
        n_ins = int(st.size[st.insert].sum())
        self.ins_keys, self.ins_vals = WG.fill_keys(cfg.seed * 1000 + 999_999, 0, n_ins, dev)
        # per-table lookup pools (keys, expected answers, outputs), arrival order; the stream's
        # read-after-write keys name flows of the insert pool that an earlier burst of the table
        # inserts, so their expected answer is that flow's value
        look = ~st.insert
        self.pools = []
        raw_bounds = np.searchsorted(st.raw_table, np.arange(cfg.n_tables + 1))  # raw_table is sorted
        for t in range(cfg.n_tables):
            n = int(st.size[look & (st.table == t)].sum())
            keys, ef, ev = WG.lookup_batch(cfg.seed * 1000 + t, n, self.warm, cfg.neg_rate, 1, device=dev)
            lo, hi = int(raw_bounds[t]), int(raw_bounds[t + 1])
            if hi > lo:
                pos = torch.from_numpy(st.raw_pos[lo:hi]).to(dev)
                src = torch.from_numpy(st.raw_src[lo:hi]).to(dev)
                keys[pos] = self.ins_keys[src]
                ef[pos] = 1
                ev[pos] = self.ins_vals[src]
            self.pools.append(dict(keys=keys, expect_found=ef, expect_value=ev,
                                   vals=torch.zeros(n, dtype=torch.int64, device=dev),
                                   found=torch.zeros(n, dtype=torch.uint8, device=dev)))
        tids = np.repeat(st.table[st.insert], st.size[st.insert]).astype(np.int32)
        self.ins_tables = torch.from_numpy(tids).to(dev)
        self.ins_status = torch.zeros(n_ins, dtype=torch.uint8, device=dev)
        self.ins_ws = torch.empty(K.ckpp_workspace_bytes(max(1, n_ins)), dtype=torch.uint8, device=dev)
        self.batch = BatchedLookup(self.tables, max_jobs=K.BATCH_MAX_JOBS, device=dev)
        torch.cuda.synchronize(dev)

    def reset_outputs(self):
        for p in self.pools:
            p["vals"].zero_()
            p["found"].zero_()
        self.ins_status.zero_()

    # ------------------------------------------------------------------ runs
    def run(self, mode: str = "batched", warmup_fraction: float = 0.1) -> dict:
        """Serve the whole stream in real time; mode 'batched' (continuous
        batching) or 'plain' (one launch per burst)."""
        cfg, st, dev = self.cfg, self.stream, self.device
        cuda = torch.cuda.current_stream(dev)
        n_bursts = st.arrival.shape[0]
        done_at = np.full(n_bursts, np.nan)
        in_flight = deque()  # (event, bursts it completes, turn or None)
        planner = TurnPlanner(st, cfg, K.BATCH_MAX_JOBS)
        nxt = 0  # plain mode: first burst not yet launched
        lib = K.library()
        # a ring of pinned job buffers: the host fills one while earlier copies are still queued
        ring = [torch.zeros(K.BATCH_MAX_JOBS * K.JOB_BYTES, dtype=torch.uint8).pin_memory() for _ in range(8)]
        ring_event = [None] * len(ring)
        slot = 0
        pools = [np.array([p[name].data_ptr() for p in self.pools], np.uint64) for name in ("keys", "vals", "found")]
        stage_args = (np.ascontiguousarray(st.table, np.uint32), np.ascontiguousarray(st.offset, np.int64),
                      np.ascontiguousarray(st.size, np.uint32), *pools)
        stage_ptrs = tuple(a.ctypes.data for a in stage_args)
        jobs_ptr = self.batch.jobs.data_ptr()
        tuning = K.ckpp_batch_tuning(*self.batch.tuning, *([0] * (4 - len(self.batch.tuning))))
        tuning_ref = ctypes.byref(tuning)
        batch_h = self.batch.handle
        handles = [t.handle for t in self.tables]
        ws_small = torch.empty(K.ckpp_workspace_bytes(cfg.max_burst), dtype=torch.uint8, device=dev)
        ins_keys, ins_vals = self.ins_keys.data_ptr(), self.ins_vals.data_ptr()
        ins_tables, ins_status = self.ins_tables.data_ptr(), self.ins_status.data_ptr()
        ins_ws, ins_ws_bytes = self.ins_ws.data_ptr(), self.ins_ws.numel()
        launches = flushes = held = 0
        starts, groups, gpu_busy = [], [], []
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(cuda)

        def retire(block: bool):
            while in_flight and (block or in_flight[0][0].query()):
                ev, idx, turn = in_flight.popleft()
                ev.synchronize()
                done_at[idx] = ev_time(ev)
                if turn is not None:
                    planner.complete(turn)
                if starts:
                    gpu_busy.append(starts.pop(0).elapsed_time(ev) / 1e3)
                block = False

        def ev_time(ev):
            return e0.elapsed_time(ev) / 1e3

        sh = cuda.cuda_stream
        while (not planner.finished() if mode == "batched" else nxt < n_bursts) or in_flight:
            retire(False)
            now = time.perf_counter() - t0
            if mode == "batched":
                action, turn, wake = planner.plan(now, bool(in_flight))
                if action == "idle":
                    if not in_flight:
                        time.sleep(max(0.0, min(50e-6, wake - now)))
                    continue
                if action == "block":
                    retire(True)
                    continue
                if action == "none":
                    continue
                look_idx = np.concatenate([turn.lookups, turn.lookups_after])
                n_first = turn.lookups.shape[0]
                nj = look_idx.shape[0]
                # the turn's host work comes first, so that its launches go out back to back
                if nj:
                    if ring_event[slot] is not None:
                        ring_event[slot].synchronize()  # the copy that last read this buffer is done
                    K._check(lib.ckpp_serve_stage_jobs(look_idx.ctypes.data, nj, *stage_ptrs, ring[slot].data_ptr()),
                             "ckpp_serve_stage_jobs")
                    nbytes_jobs = nj * K.JOB_BYTES
                    self.batch.jobs[:nbytes_jobs].copy_(ring[slot][:nbytes_jobs], non_blocking=True)
                ev_start = torch.cuda.Event(enable_timing=True)
                ev_start.record(cuda)
                # 1. lookups whose table has no waiting insert (the job count is known here: the
                #    prefix scan is sized to it, no device count)
                if n_first:
                    K._check(lib.ckpp_batch_lookup(batch_h, jobs_ptr, n_first, None, 0, tuning_ref, sh),
                             "ckpp_batch_lookup")
                    launches += 1
                # 2. the waiting inserts, one contiguous range of the insert pool
                if turn.inserts:
                    first = turn.insert_first
                    K._check(lib.ckpp_batch_insert(batch_h, ins_keys + 16 * first, ins_tables + 4 * first,
                                                   ins_vals + 8 * first, turn.insert_keys, 0, 0, ins_status + first,
                                                   ins_ws, ins_ws_bytes, sh), "ckpp_batch_insert")
                    launches += 1
                    flushes += 1
                # 3. lookups held behind those inserts
                if nj > n_first:
                    K._check(lib.ckpp_batch_lookup(batch_h, jobs_ptr + n_first * K.JOB_BYTES, nj - n_first, None, 0,
                                                   tuning_ref, sh), "ckpp_batch_lookup")
                    launches += 1
                    held += nj - n_first
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(cuda)
                if nj:
                    ring_event[slot] = ev
                    slot = (slot + 1) % len(ring)
                in_flight.append((ev, turn.done, turn))
                starts.append(ev_start)
                groups.append(turn.admitted.stop - turn.admitted.start)
            elif nxt < n_bursts and st.arrival[nxt] <= now:  # plain: one launch per burst, as it arrives
                hi = int(np.searchsorted(st.arrival, now, side="right"))
                for b in range(nxt, hi):
                    t = int(st.table[b])
                    n = int(st.size[b])
                    off = int(st.offset[b])
                    if st.insert[b]:
                        lib.ckpp_bulk_insert(handles[t], self.ins_keys[off:].data_ptr(),
                                             self.ins_vals[off:].data_ptr(), n, 0, 0,
                                             self.ins_status[off:].data_ptr(), ws_small.data_ptr(),
                                             ws_small.numel(), sh)
                    else:
                        p = self.pools[t]
                        lib.ckpp_bulk_lookup(handles[t], p["keys"][off:].data_ptr(), n, p["vals"][off:].data_ptr(),
                                             p["found"][off:].data_ptr(), 0, 0, sh)
                    launches += 1
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(cuda)
                in_flight.append((ev, np.arange(nxt, hi), None))
                nxt = hi
            elif not in_flight and nxt < n_bursts:
                time.sleep(max(0.0, min(50e-6, st.arrival[nxt] - now)))
        retire(True)
        wall = time.perf_counter() - t0
        lat = (done_at - st.arrival) * 1e6
        keep = st.arrival >= warmup_fraction * cfg.duration_s
        lk = ~st.insert
        served = int(st.size[lk].sum())
        return {
            "mode": mode, "bursts": int(n_bursts), "lookups": served, "inserts": int(st.size[st.insert].sum()),
            "offered_glookups": round(served / cfg.duration_s / 1e9, 3),
            "achieved_glookups": round(served / wall / 1e9, 3), "wall_s": round(wall, 4),
            "launches": launches,
            "groups": len(groups) if groups else None,
            "bursts_per_group": round(float(np.mean(groups)), 1) if groups else None,
            "gpu_busy_fraction": round(float(np.sum(gpu_busy)) / wall, 3) if gpu_busy else None,
            "gpu_ms_per_group": round(float(np.mean(gpu_busy)) * 1e3, 4) if gpu_busy else None,
            "latency_us": percentiles(lat[keep]),
            "lookup_latency_us": percentiles(lat[keep & lk]),
            "insert_latency_us": percentiles(lat[keep & st.insert]),
            "insert_flushes": flushes if mode == "batched" else None,
            "held_lookup_bursts": held if mode == "batched" else None,
            "read_after_write_keys": int(st.raw_pos.shape[0]),
        }

    def check(self) -> dict:
        """Every lookup output equals the sequential answer (the warm fill's map
        plus the flows inserted by earlier bursts of the same table); every
        insert status is INSERTED."""
        ok_lookups = all(bool(torch.equal(p["found"], p["expect_found"])) and
                         bool(torch.equal(p["vals"], p["expect_value"])) for p in self.pools)
        ok_inserts = bool((self.ins_status == K.ST_INSERTED).all())
        return {"lookups_match_map": ok_lookups, "inserts_all_inserted": ok_inserts}
