"""Served form: a continuous-batching request loop over device-resident tables.

Packet bursts arrive from many ports (``serve_policy.draw_stream``). The loop
runs in real time on the host, as native code (``ckpp_serve_run`` of
include/ckpp_serve.h):

* it retires finished turns (CUDA event queries) and frees their staging
  footprint;
* it asks the turn planner (admission within an HBM footprint budget, write
  coalescing, per-table arrival order) what to launch;
* it launches that without waiting for the previous turn, all on one stream,
  in the turn's order: the lookups whose table has no waiting insert as one
  persistent ``ckpp_batch_lookup`` (one job per burst); when the planner
  flushes them, the waiting inserts as one multi-table ``ckpp_batch_insert``
  (an insert call has a fixed cost of several dependent kernels, so
  coalescing writes keeps that cost from every turn); then the lookups that
  were held behind those inserts as a second batched lookup.

Each table applies its lookups and inserts in arrival order (the planner's
rule), so every burst gets the result it gets when every burst runs alone in
arrival order. Lookups read flows of the warm fill, unknown flows, and (a
``raw_fraction`` of their keys) flows inserted by earlier insert bursts of
the same table during the run; the tests compare every result with that
sequential answer. Per-burst latency is completion time (the turn's CUDA
event on the device clock, from an event recorded at the start) minus arrival
time.

The comparison arm serves the same arrival stream with one plain launch per
burst (``ckpp_bulk_lookup`` / ``ckpp_bulk_insert``) as bursts arrive
(``ckpp_serve_run_plain``, also native).
"""

from __future__ import annotations

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
        # a second descriptor for the second stream's lookups (overlap): a descriptor's launches must not overlap
        self.batch_b = BatchedLookup(self.tables, max_jobs=1, device=dev) if cfg.overlap else None
        torch.cuda.synchronize(dev)

    def reset_outputs(self):
        for p in self.pools:
            p["vals"].zero_()
            p["found"].zero_()
        self.ins_status.zero_()

    # ------------------------------------------------------------------ runs
    def run(self, mode: str = "batched", warmup_fraction: float = 0.1) -> dict:
        """Serve the whole stream in real time; mode 'batched' (continuous
        batching, ckpp_serve_run) or 'plain' (one launch per burst,
        ckpp_serve_run_plain). Both loops are native host code driving the
        device on the current stream."""
        import ctypes as C

        cfg, st, dev = self.cfg, self.stream, self.device
        cuda = torch.cuda.current_stream(dev)
        n_bursts = st.arrival.shape[0]
        planner = TurnPlanner(st, cfg, K.BATCH_MAX_JOBS)
        ring_slots = 8
        h_jobs = torch.zeros(ring_slots * K.BATCH_MAX_JOBS * K.JOB_BYTES, dtype=torch.uint8).pin_memory()
        pools = [np.array([p[name].data_ptr() for p in self.pools], np.uint64) for name in ("keys", "vals", "found")]
        # with overlap every turn reads its own ring slot of device job records
        d_jobs = (torch.empty(ring_slots * K.BATCH_MAX_JOBS * K.JOB_BYTES, dtype=torch.uint8, device=dev)
                  if cfg.overlap else self.batch.jobs)
        buf = K.ckpp_serve_buffers(
            pools[0].ctypes.data, pools[1].ctypes.data, pools[2].ctypes.data, cfg.n_tables, K.BATCH_MAX_JOBS,
            self.ins_keys.data_ptr(), self.ins_tables.data_ptr(), self.ins_vals.data_ptr(),
            self.ins_status.data_ptr(), self.ins_ws.data_ptr(), self.ins_ws.numel(), d_jobs.data_ptr(),
            h_jobs.data_ptr(), ring_slots, cfg.max_inflight, self.batch_b.handle if self.batch_b else None)
        done_at = np.full(n_bursts, np.nan)
        stats = K.ckpp_serve_stats()
        lib = K.library()
        torch.cuda.synchronize(dev)
        if mode == "batched":
            tn = self.batch.tuning
            tuning = K.ckpp_batch_tuning(tn[0], tn[1], tn[2], tn[3] if len(tn) > 3 else 0)
            rc = lib.ckpp_serve_run(planner._h, self.batch.handle, C.byref(buf), C.byref(tuning), cuda.cuda_stream,
                                    done_at.ctypes.data, C.byref(stats))
            K._check(rc, "ckpp_serve_run")
        else:
            handles = (C.c_void_p * cfg.n_tables)(*[t.handle for t in self.tables])
            rc = lib.ckpp_serve_run_plain(planner._h, handles, C.byref(buf), cuda.cuda_stream, done_at.ctypes.data,
                                          C.byref(stats))
            K._check(rc, "ckpp_serve_run_plain")
        torch.cuda.synchronize(dev)
        del pools, h_jobs, d_jobs
        if np.isnan(done_at).any():
            raise RuntimeError(f"{int(np.isnan(done_at).sum())} bursts were never completed")
        wall = stats.wall_s
        lat = (done_at - st.arrival) * 1e6
        keep = st.arrival >= warmup_fraction * cfg.duration_s
        lk = ~st.insert
        served = int(st.size[lk].sum())
        turns = int(stats.turns)
        return {
            "mode": mode, "bursts": int(n_bursts), "lookups": served, "inserts": int(st.size[st.insert].sum()),
            "offered_glookups": round(served / cfg.duration_s / 1e9, 3),
            "achieved_glookups": round(served / wall / 1e9, 3), "wall_s": round(wall, 4),
            "launches": int(stats.launches),
            "groups": turns,
            "bursts_per_group": round(int(stats.admitted) / turns, 1) if turns else None,
            "gpu_busy_fraction": round(stats.gpu_busy_s / wall, 3) if wall else None,
            "gpu_ms_per_group": round(stats.gpu_busy_s / turns * 1e3, 4) if turns else None,
            "latency_us": percentiles(lat[keep]),
            "lookup_latency_us": percentiles(lat[keep & lk]),
            "insert_latency_us": percentiles(lat[keep & st.insert]),
            "insert_flushes": int(stats.flushes) if mode == "batched" else None,
            "held_lookup_bursts": int(stats.held) if mode == "batched" else None,
            "overlap": bool(cfg.overlap) if mode == "batched" else None,
            "trailing_lookup_bursts": int(stats.trailing) if mode == "batched" and cfg.overlap else None,
            "gpu_busy_second_stream_fraction": (round(stats.gpu_busy_b_s / wall, 3)
                                                if mode == "batched" and cfg.overlap and wall else None),
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
