"""Bulk-lookup throughput of the GB300 Cuckoo++ table.

Workload (the at-scale configuration): 2^24 buckets x 8 slots (134,217,728
slots) filled to load factor 0.9 with 120,795,955 random 5-tuple keys (value =
insertion index), then bulk_lookup batches of 2^24 keys with each key negative
with probability 0.5 (Bernoulli), positives drawn uniformly from the inserted
keys. A step is one bulk_lookup of one such batch, inputs resident in HBM.
The table (4.3 GB) and the key batch (256 MB) are both larger than L2, so no
L2 flush is needed between steps.

One JSON line on rank 0. Beside the headline `value` it reports:
  e2e        the same lookups through the C ABI from pinned host buffers, the
             host->device key copy and device->host result copies timed inside;
  roofline   algorithmic bytes of the lookup kernel (32 B per bucket sector and
             per key/value record the method reads, counted on the batch by the
             library's probe-count kernel, plus 25 B of key/result streaming)
             over its measured duration, against the measured HBM copy peak;
  pos / neg  the same measurement on all-positive and all-negative batches;
  at_100M_entries  the same measurement on the same table when the fill stands at exactly
             100,000,000 entries (LF 0.745);
  mutations  bulk_insert / bulk_delete / expire throughput on the same table;
  small_config  the small configuration (2^17 buckets x 8, LF 0.9, 1M-key
             batch), L2-resident, against the measured L2 read bandwidth;
  sharding   the device half of a hash-sharded lookup of the same batch over 8
             shards (partition by owner, results back in the caller's order),
             beside one local lookup;
  cpu_baseline  the CPU oracle's lookup rate on a bounded sample (rank 0, N=1).

--impl reference times the CPU oracle itself (the reference arm of this
build): it builds the oracle table of the same workload and times its lookups,
each step a bounded sample.

Multi-GPU (torchrun): every rank builds and serves its own table (independent,
share-nothing tables as in the paper's multi-core setting), no collective on
the data path; value = lookups of all ranks / max time over ranks.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Glookups/s at 100M entries LF0.9 (pos/neg), % of random-access HBM roofline"
UNIT = "Glookups/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--log2-buckets", type=int, default=24)
    p.add_argument("--load-factor", type=float, default=0.9)
    p.add_argument("--neg-rate", type=float, default=0.5)
    p.add_argument("--log2-batch", type=int, default=24)
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-side", action="store_true", help="skip pos/neg/e2e/mutation side measurements")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU oracle timing budget")
    p.add_argument("--workload", default="scale",
                   choices=["scale", "batched", "sweep", "served", "mixed", "insert"],
                   help="scale: the headline at-scale lookup (default); batched: many tables in one launch vs "
                        "one launch per table; sweep: load factor x negative rate x lookup strategy grid; "
                        "served: continuous-batching "
                        "request loop vs one launch per burst; mixed: insert/lookup/delete/expire mix on a "
                        "200M-slot table with timers; insert: bulk insert rate as a table fills from LF 0.85 "
                        "to 0.99")
    p.add_argument("--mixed-batches", type=int, default=400, help="mixed: batches (time units) to run")
    p.add_argument("--serve-seconds", type=float, default=0.2, help="served: seconds of offered traffic")
    p.add_argument("--serve-modes", default="batched,plain", help="served: arms to run")
    p.add_argument("--serve-max-inflight", type=int, default=None,
                   help="served: turns queued on the device at most (0: no limit)")
    p.add_argument("--serve-one-stream", action="store_true",
                   help="served: flushes on the lookups' stream (default: on a second stream, beside later turns)")
    p.add_argument("--serve-flush-keys", type=int, default=None,
                   help="served: coalesced inserts go out once this many keys wait (default: the loop's own)")
    p.add_argument("--serve-flush-us", type=float, default=None,
                   help="served: ... or once the oldest waiting insert burst is this old")
    p.add_argument("--serve-hold-us", type=float, default=None,
                   help="served: ... or once a lookup held behind waiting inserts is this old")
    p.add_argument("--tables", type=int, default=4096, help="batched: number of tables")
    p.add_argument("--record-traffic", metavar="CSV", default=None,
                   help="write profiles/lookup_traffic.json from an ncu --csv log of the lookup kernel and exit")
    return p.parse_args()


# ------------------------------------------------------------------ helpers

NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e datasheet figure, reported beside the measured copy peak


L2_BYTES = 129 << 20  # GB300 L2 (about 129 MB)
TRAFFIC_CONFIG = (24, 24, 0.9, 0.5)  # the captured traffic's log2 buckets, log2 batch, LF, negative rate


def scale_config(args, n_fill: int) -> dict:
    """The config block of the at-scale lookup, shared by both arms."""
    nb, n = 1 << args.log2_buckets, 1 << args.log2_batch
    table_bytes = 256 + nb * 256
    size = f"{n >> 20}M" if n >= 1 << 20 and n % (1 << 20) == 0 else str(n)
    if table_bytes > L2_BYTES and n * 16 > L2_BYTES:
        l2 = f"inputs larger than L2 (table {table_bytes / 1e9:.1f} GB, keys {n * 16 / 2**20:.0f} MB); no flush"
    else:
        l2 = f"inputs not larger than L2 (table {table_bytes / 2**20:.0f} MB, keys {n * 16 / 2**20:.1f} MB); no flush"
    return {"workload": f"plain Cuckoo++ at scale: 2^{args.log2_buckets} buckets x 8 slots, LF {args.load_factor}, "
                        f"{size}-key bulk_lookup",
            "n_buckets": nb, "slots": 8, "entries": n_fill, "load_factor": args.load_factor, "batch": n,
            "neg_rate": args.neg_rate, "timers": False, "l2": l2}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


LOOKUP_SOURCES = ("paper_1712_09624_gb300/csrc/lookup.cu", "paper_1712_09624_gb300/csrc/probe.cuh",
                  "paper_1712_09624_gb300/csrc/ckpp_device.cuh")


def sources_sha256(paths=LOOKUP_SOURCES) -> str:
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def alg_bytes_of(counts, n: int) -> float:
    """Algorithmic bytes of a lookup batch from its read counts (primary
    bucket reads, secondary bucket reads, record reads, second-line reads):
    32 bytes per bucket read (tags, filter, busy mask) and per record read
    (key and value), plus 16 bytes of key in and 9 of result out per lookup.
    The count is the method's, independent of how the layout groups fields
    into lines."""
    return 32.0 * float(counts[0] + counts[1] + counts[2]) + 25.0 * n


def line_bytes_of(counts, n: int) -> float:
    """Bytes a lookup batch moves as whole 128-byte lines (one per line
    request) plus its 16 bytes of key in and 9 of result out per lookup."""
    return 128.0 * lines_of(counts) + 25.0 * n


def lines_of(counts) -> float:
    """128-byte line requests a lookup batch makes: one per bucket read, plus
    one per second-line read."""
    return float(counts[0] + counts[1] + counts[3])


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "lookup_traffic.json")


def profiled_traffic():
    """Per-launch DRAM bytes of the lookup kernel from the committed capture
    (profiles/lookup_traffic.json, written by --record-traffic), if it was
    taken on the current kernel sources (sha256 over the files the kernel is
    built from), else None."""
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)
        current = sources_sha256(tuple(d["sources"]))
    except (OSError, ValueError, KeyError):
        return None
    if d.get("sources_sha256") != current:
        return None
    return float(d["traffic_bytes_per_launch"])


# ncu's unit spellings -> bytes, or microseconds for times
_UNIT_SCALE = {"byte": 1, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9, "tbyte": 1e12,
               "nsecond": 1e-3, "usecond": 1.0, "msecond": 1e3, "second": 1e6,
               "ns": 1e-3, "us": 1.0, "ms": 1e3, "s": 1e6}


def record_traffic(csv_path: str):
    """Write profiles/lookup_traffic.json from an ncu --csv log of the lookup
    kernel with dram__bytes_read.sum, dram__bytes_write.sum and
    gpu__time_duration.sum (the first captured launch), stamped with the
    sha256 of the current kernel sources."""
    import csv
    rows = list(csv.DictReader(line for line in open(csv_path) if line.startswith('"')))
    rows = [r for r in rows if "lookup_kernel" in r.get("Kernel Name", "")]
    if not rows:
        raise SystemExit(f"{csv_path}: no lookup_kernel rows")
    first = rows[0]["ID"]
    m = {}
    for r in rows:
        if r["ID"] == first:
            m[r["Metric Name"]] = float(r["Metric Value"].replace(",", "")) * _UNIT_SCALE[r["Metric Unit"].lower()]
    rd, wr = m["dram__bytes_read.sum"], m["dram__bytes_write.sum"]
    d = {"kernel": rows[0]["Kernel Name"],
         "config": dict(zip(("log2_buckets", "log2_batch", "load_factor", "neg_rate"), TRAFFIC_CONFIG)),
         "traffic_bytes_per_launch": int(round(rd + wr)), "dram_bytes_read": int(round(rd)),
         "dram_bytes_write": int(round(wr)), "gpu_time_us": round(m["gpu__time_duration.sum"], 2),
         "sources": list(LOOKUP_SOURCES), "sources_sha256": sources_sha256(),
         "command": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
                    "--clock-control none -k regex:lookup_kernel -s 2 -c 1 --csv --log-file traffic.csv "
                    "python bench.py --steps 20 --warmup 3 --no-cpu-baseline --no-side; "
                    "python bench.py --record-traffic traffic.csv"}
    with open(TRAFFIC_FILE, "w") as f:
        json.dump(d, f, indent=1)
        f.write("\n")
    print(json.dumps(d))


class ClockSampler:
    """nvidia-smi clock/throttle samples with host timestamps."""

    QUERY = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            return self
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), [x.strip() for x in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)

    def summary(self, t0: float, t1: float):
        inside = [s for t, s in self.samples if t0 <= t <= t1]
        window = "timed"
        if not inside:
            inside = [s for t, s in self.samples if t <= t1]
            window = "before-and-during"
        if not inside:
            return None
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(s[0]) for s in inside if num(s[0]) is not None]
        mx = [num(s[1]) for s in inside if num(s[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in inside for i in range(4) if len(s) > 4 + i and "Active" in s[4 + i]
                          and "Not" not in s[4 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside), "window": window}


# ------------------------------------------------------------- our arm

def lookup_side(args, K, W, table, fill, m, n, seed, dev, stream, steps=20, warmup=3):
    """Lookups on the table as it stands with the first m fill keys inserted:
    a checked, timed n-key batch (negative rate as the headline) drawn from
    those keys, with its algorithmic bytes and line requests."""
    import torch
    sub = W.FillWorkload(fill.keys[:m], fill.values[:m])
    q = W.lookup_batch(seed, n, sub, args.neg_rate, batch_id=100)
    kk = torch.from_numpy(q.keys).to(dev)
    ov = torch.empty(n, dtype=torch.int64, device=dev)
    of = torch.empty(n, dtype=torch.bool, device=dev)
    K.ckpp_bulk_lookup(table.handle, kk, ov, of, 0, 0, stream)
    torch.cuda.synchronize()
    exact = bool((of.cpu().numpy() == q.expect_found).all()) and \
        bool((ov.cpu().numpy().view(np.uint64) == q.expect_value).all())
    c = table.probe_counts(kk).cpu().numpy()
    for _ in range(warmup):
        K.ckpp_bulk_lookup(table.handle, kk, ov, of, 0, 0, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        K.ckpp_bulk_lookup(table.handle, kk, ov, of, 0, 0, stream)
    e1.record(stream)
    e1.synchronize()
    per = e0.elapsed_time(e1) / 1e3 / steps
    peak, _ = measured_peaks()
    return {"entries": m, "load_factor": round(m / (8 * table.n_buckets), 4), "value": round(n / per / 1e9, 4),
            "unit": UNIT, "neg_rate": args.neg_rate, "exact": exact,
            "alg_bytes_per_lookup": round(alg_bytes_of(c, n) / n, 3),
            "frac": round(alg_bytes_of(c, n) / per / 1e9 / peak, 4),
            "line_requests_per_lookup": round(lines_of(c) / n, 5)}


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1712_09624_gb300 import _ckpp as K
    from paper_1712_09624_gb300 import dist as D
    from paper_1712_09624_gb300 import workload as W
    from paper_1712_09624_gb300.table import FlowTable

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    nb = 1 << args.log2_buckets
    n_fill = int(args.load_factor * nb * 8)
    n = 1 << args.log2_batch
    seed = D.rank_seed(args.seed, rank)  # independent tables per rank
    stream = torch.cuda.current_stream()

    fill = W.fill(seed, n_fill)
    table = FlowTable(nb, timers=False, seed=seed, device=dev)
    chunk = 1 << 24
    ins_times = []
    # the fill stops once at exactly 100,000,000 entries (LF 0.745 on 2^27 slots) for a side measurement
    stop_100m = 100_000_000 if (rank == 0 and not args.no_side and n_fill > 100_000_000) else None
    bounds = sorted(set(list(range(0, n_fill, chunk)) + ([stop_100m] if stop_100m else [])) | {n_fill})
    at_100m = None
    for lo, hi in zip(bounds[:-1], bounds[1:]):
        if lo == stop_100m:
            at_100m = lookup_side(args, K, W, table, fill, lo, n, seed, dev, stream)
        k = torch.from_numpy(fill.keys[lo:hi]).to(dev)
        v = torch.from_numpy(fill.values[lo:hi].view(np.int64)).to(dev)
        st = torch.empty(k.shape[0], dtype=torch.uint8, device=dev)
        ws = table.workspace(k.shape[0])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        K.ckpp_bulk_insert(table.handle, k, v, st, ws, 0, 0, stream)
        e1.record(stream)
        e1.synchronize()
        ins_times.append((k.shape[0], e0.elapsed_time(e1) / 1e3))
        if not bool((st == K.ST_INSERTED).all()):
            raise RuntimeError("fill reported a status other than INSERTED")
    if table.sync_status() != 0:
        raise RuntimeError("device wait gave up during the fill")

    def batch(neg, bid):
        q = W.lookup_batch(seed, n, fill, neg, batch_id=bid)
        return q, torch.from_numpy(q.keys).to(dev)

    q, keys = batch(args.neg_rate, 0)
    out_v = torch.empty(n, dtype=torch.int64, device=dev)
    out_f = torch.empty(n, dtype=torch.bool, device=dev)

    def lookup(kk, ov, of):
        K.ckpp_bulk_lookup(table.handle, kk, ov, of, 0, 0, stream)

    # correctness of the timed configuration against the map definition
    lookup(keys, out_v, out_f)
    torch.cuda.synchronize()
    if not (out_f.cpu().numpy() == q.expect_found).all() or \
            not (out_v.cpu().numpy().view(np.uint64) == q.expect_value).all():
        raise RuntimeError("lookup results differ from the workload's key -> value map")
    counts = table.probe_counts(keys).cpu().numpy()
    alg_bytes = alg_bytes_of(counts, n)

    def timed(kk, ov, of, steps, warmup):
        for _ in range(warmup):
            lookup(kk, ov, of)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.time()
        e0.record(stream)
        for _ in range(steps):
            lookup(kk, ov, of)
        e1.record(stream)
        e1.synchronize()
        t1 = time.time()
        if world > 1:
            torch.distributed.barrier()
        return e0.elapsed_time(e1) / 1e3, t0, t1

    sampler = ClockSampler(local_rank).start() if rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    secs, t0, t1 = timed(keys, out_v, out_f, args.steps, args.warmup)
    time.sleep(0.15 if sampler else 0)
    if sampler:
        sampler.stop()
    secs = D.max_over_ranks(secs, dev)
    per_launch = secs / args.steps
    value = D.job_throughput(n, args.steps, secs, world) / 1e9

    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / per_launch / 1e9
    # the committed capture is of the default configuration only
    same = (args.log2_buckets, args.log2_batch, args.load_factor, args.neg_rate) == TRAFFIC_CONFIG
    traffic = profiled_traffic() if same else None
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": scale_config(args, n_fill),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "peak_kind": f"{peak_kind} copy bandwidth",
                     "alg_bytes_per_lookup": round(alg_bytes / n, 3),
                     "reads_per_lookup": {"primary": float(counts[0] / n), "secondary": float(counts[1] / n),
                                          "record": float(counts[2] / n)},
                     "line_requests_per_lookup": round(lines_of(counts) / n, 5),
                     "nominal_peak_GBs": NOMINAL_HBM_GBS,
                     "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                     "whole_lines": {"bytes_per_lookup": round(line_bytes_of(counts, n) / n, 2),
                                     "frac": round(line_bytes_of(counts, n) / per_launch / 1e9 / peak, 4),
                                     "note": "the bytes the kernel moves: 128 B per line request plus 25 B "
                                             "of keys and results; frac above counts the method's bytes"}},
        "gpu_launches": args.steps,
    }
    if sampler:
        out["clocks"] = sampler.summary(t0, t1)

    if rank == 0 and not args.no_side:
        side = {}
        for name, neg in (("pos", 0.0), ("neg", 1.0)):
            qq, kk = batch(neg, 1 + int(neg))
            s, _, _ = timed(kk, out_v, out_f, max(10, args.steps // 4), 3)
            c = table.probe_counts(kk).cpu().numpy()
            b = alg_bytes_of(c, n)
            side[name] = {"value": round(n * max(10, args.steps // 4) / s / 1e9, 4), "unit": UNIT,
                          "alg_bytes_per_lookup": round(b / n, 3),
                          "line_requests_per_lookup": round(lines_of(c) / n, 5),
                          "frac": round(b / (s / max(10, args.steps // 4)) / 1e9 / peak, 4)}
        out.update(side)
        if at_100m:
            out["at_100M_entries"] = at_100m
        out["e2e"] = e2e_lookup(args, table, q, dev, stream)
        out["mutations"] = mutation_rates(table, dev, stream, ins_times, seed)
        out["small_config"] = small_config(args, dev, stream)
        out["sharding"] = shard_side(args, keys, per_launch, dev, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, fill, q, nb, seed)
        out["cpu_baseline_all_cores"] = cpu_baseline_share_nothing(args)
    return out


def shard_side(args, keys, lookup_s, dev, stream, n_shards: int = 8, steps: int = 10):
    """The device half of a hash-sharded lookup on the headline batch, as if
    over 8 GPUs: partition the 16M keys by owner (ckpp_shard_partition: the
    owner-sorted keys and the order) and put the results back in the caller's
    order (ckpp_shard_unpermute of the 8-byte values and the flags). Timed by
    CUDA events (mean of `steps` after 3 warm-ups) and set against one local
    lookup of the same batch. The all-to-alls between the two are not
    measured (one GPU); their volume is stated."""
    import torch

    from paper_1712_09624_gb300 import _ckpp as K
    n = keys.shape[0]
    ws = torch.empty(K.ckpp_shard_workspace_bytes(n, n_shards), dtype=torch.uint8, device=dev)
    pos = torch.empty(n, dtype=torch.int32, device=dev)
    keys_s = torch.empty((n, 16), dtype=torch.uint8, device=dev)
    counts = torch.empty(n_shards, dtype=torch.int64, device=dev)
    vals_in = torch.arange(n, dtype=torch.int64, device=dev)
    flags_in = torch.ones(n, dtype=torch.uint8, device=dev)
    vals_out = torch.empty_like(vals_in)
    flags_out = torch.empty_like(flags_in)

    def part():
        K.ckpp_shard_partition(keys, None, args.seed, n_shards, pos, keys_s, None, counts, ws, stream)

    def unperm():
        K.ckpp_shard_unpermute(pos, vals_in, flags_in, vals_out, flags_out, stream)

    def time_of(fn):
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3 / steps

    tp, tu = time_of(part), time_of(unperm)
    c = counts.cpu().numpy()
    # unpermute gathers out[i] = in[pos[i]]: with vals_in = arange, vals_out is pos, a permutation, so every
    # index appears once
    ok = int(c.sum()) == n and bool(torch.bincount(vals_out, minlength=n).eq(1).all()) and bool(flags_out.all())
    return {"n_shards": n_shards, "partition_us": round(tp * 1e6, 1), "unpermute_us": round(tu * 1e6, 1),
            "local_lookup_us": round(lookup_s * 1e6, 1),
            "device_overhead_vs_lookup": round((tp + tu) / lookup_s, 3),
            "largest_shard_share": round(float(c.max()) / n, 5), "consistent": ok,
            "all_to_all_bytes_per_key": {"keys_out": 16, "results_back": 9},
            "note": "one GPU: the partition and unpermute kernels only; the two all-to-alls are not measured"}


def l2_read_peak(dev, stream, mib: int = 48, passes: int = 20, steps: int = 10):
    """Streaming read bandwidth of a buffer that sits in L2 (the L2 read probe
    of the workload library, 16-byte ld.global.cg loads), by CUDA events:
    bytes x passes per launch over the launch time, best of `steps` launches
    after 3 warm-ups."""
    import torch

    from paper_1712_09624_gb300 import workload_gpu as WG
    buf = torch.ones(mib << 20, dtype=torch.uint8, device=dev)
    sink = torch.zeros(1, dtype=torch.int64, device=dev)
    for _ in range(3):
        WG.l2_read(buf, passes, sink, stream)
    best = None
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        WG.l2_read(buf, passes, sink, stream)
        e1.record(stream)
        e1.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        best = sec if best is None else min(best, sec)
    return (mib << 20) * passes / best / 1e9


def small_config(args, dev, stream, steps: int = 200, warmup: int = 5):
    """The small configuration: 2^17 buckets x 8 slots filled to LF 0.9
    (943,718 keys), one 2^20-key lookup batch with 50% negatives. The table
    (32 MiB), the keys (16 MiB) and the results (9 MiB) all sit in L2, so the
    batch is measured against the L2 read bandwidth (measured here by the L2
    read probe) rather than the HBM copy peak. Results are checked against the
    workload's key -> value map."""
    import torch

    from paper_1712_09624_gb300 import _ckpp as K
    from paper_1712_09624_gb300 import workload as W
    from paper_1712_09624_gb300.table import FlowTable
    nb, lf, n, neg = 1 << 17, 0.9, 1 << 20, 0.5
    fill = W.fill(args.seed, int(lf * nb * 8))
    t = FlowTable(nb, seed=args.seed, device=dev)
    st = t.insert(fill.keys, fill.values, 0, 0, stream)
    q = W.lookup_batch(args.seed, n, fill, neg)
    kk = torch.from_numpy(q.keys).to(dev)
    ov = torch.empty(n, dtype=torch.int64, device=dev)
    of = torch.empty(n, dtype=torch.bool, device=dev)
    K.ckpp_bulk_lookup(t.handle, kk, ov, of, 0, 0, stream)
    torch.cuda.synchronize()
    exact = bool((st == K.ST_INSERTED).all()) and bool((of.cpu().numpy() == q.expect_found).all()) and \
        bool((ov.cpu().numpy().view(np.uint64) == q.expect_value).all())
    c = t.probe_counts(kk).cpu().numpy()
    for _ in range(warmup):
        K.ckpp_bulk_lookup(t.handle, kk, ov, of, 0, 0, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        K.ckpp_bulk_lookup(t.handle, kk, ov, of, 0, 0, stream)
    e1.record(stream)
    e1.synchronize()
    per = e0.elapsed_time(e1) / 1e3 / steps
    l2 = l2_read_peak(dev, stream)
    hbm, _ = measured_peaks()
    b = alg_bytes_of(c, n)
    return {"workload": "plain Cuckoo++ small: 2^17 buckets x 8 slots, LF 0.9, 1M-key bulk_lookup, 50% negative",
            "value": round(n / per / 1e9, 4), "unit": UNIT, "steps": steps, "ms_per_step": round(per * 1e3, 5),
            "exact": exact, "l2": "table, keys and results L2-resident; no flush",
            "alg_bytes_per_lookup": round(b / n, 3), "line_requests_per_lookup": round(lines_of(c) / n, 5),
            "roofline": {"bound": "l2", "achieved": round(b / per / 1e9, 1), "peak": round(l2, 1), "unit": "GB/s",
                         "frac": round(b / per / 1e9 / l2, 4),
                         "peak_kind": "measured L2 streaming read (ckpp_wl_l2_read, 48 MiB buffer, 20 passes, "
                                      "best of 10 launches)",
                         "whole_lines_frac": round(line_bytes_of(c, n) / per / 1e9 / l2, 4),
                         "frac_of_hbm_copy": round(b / per / 1e9 / hbm, 4)}}


def e2e_lookup(args, table, q, dev, stream):
    """Lookups through the C ABI with HOST buffers: the keys sit in pinned host
    memory and the results go to pinned host memory. ckpp_bulk_lookup reads and
    writes them in place over NVLink-C2C, so every step moves 16 B per key
    host->device and 9 B per key device->host inside the timed region. The
    staged variant (explicit copies around a device-buffer lookup) is reported
    beside it."""
    import torch

    from paper_1712_09624_gb300 import _ckpp as K
    n = q.keys.shape[0]
    h_keys = torch.from_numpy(q.keys).pin_memory()
    h_vals = torch.empty(n, dtype=torch.int64).pin_memory()
    h_found = torch.empty(n, dtype=torch.bool).pin_memory()
    steps = max(5, args.steps // 10)

    def run(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3

    def zero_copy():
        K.ckpp_bulk_lookup(table.handle, h_keys, h_vals, h_found, 0, 0, stream)

    secs = run(zero_copy)
    ok = bool((h_found.numpy() == q.expect_found).all()) and \
        bool((h_vals.numpy().view(np.uint64) == q.expect_value).all())
    d_keys = torch.empty((n, 16), dtype=torch.uint8, device=dev)
    d_vals = torch.empty(n, dtype=torch.int64, device=dev)
    d_found = torch.empty(n, dtype=torch.bool, device=dev)

    def staged():
        d_keys.copy_(h_keys, non_blocking=True)
        K.ckpp_bulk_lookup(table.handle, d_keys, d_vals, d_found, 0, 0, stream)
        h_vals.copy_(d_vals, non_blocking=True)
        h_found.copy_(d_found, non_blocking=True)

    secs_staged = run(staged)
    # the ceiling: the same host I/O (key in, value and flag out, same access
    # pattern) with no table behind it
    from paper_1712_09624_gb300 import workload_gpu as WG
    secs_io = run(lambda: WG.host_io(h_keys, h_vals, h_found, stream))
    link = n * steps / secs_io / 1e9
    value = n * steps / secs / 1e9
    return {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 16 * n,
            "d2h_bytes_per_step": 9 * n, "steps": steps, "results_match": ok,
            "path": "ckpp_bulk_lookup on pinned host buffers (in-place over NVLink-C2C)",
            "staged_copies_value": round(n * steps / secs_staged / 1e9, 4),
            "host_io_only_value": round(link, 4), "frac_of_host_io_only": round(value / link, 4),
            "host_io_only_note": "ckpp_wl_host_io on the same pinned buffers: each key read and its value "
                                 "and flag written over NVLink-C2C, no table"}


def mutation_rates(table, dev, stream, ins_times, seed):
    """Insert (during the fill), delete and expire rates on the same table."""
    import torch

    from paper_1712_09624_gb300 import workload as W
    from paper_1712_09624_gb300.table import FlowTable
    n_ins = sum(c for c, _ in ins_times)
    t_ins = sum(s for _, s in ins_times)
    out = {"insert_fill_Mops": round(n_ins / t_ins / 1e6, 1)}
    # delete + reinsert of 1M resident keys
    fill_keys = W.make_keys(seed, W.STREAM_INSERT_KEYS, 1 << 20)
    k = torch.from_numpy(fill_keys).to(dev)
    vals = torch.arange(k.shape[0], dtype=torch.int64, device=dev)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record(stream)
    st = table.delete(k, 0, stream)
    e[1].record(stream)
    st2 = table.insert(k, vals, 0, 0, stream)
    e[2].record(stream)
    e[2].synchronize()
    out["delete_Mops"] = round(k.shape[0] / (e[0].elapsed_time(e[1]) / 1e3) / 1e6, 1)
    out["insert_at_lf0.9_Mops"] = round(k.shape[0] / (e[1].elapsed_time(e[2]) / 1e3) / 1e6, 1)
    out["delete_ok"] = bool((st == 4).all())
    out["reinsert_ok"] = bool((st2 == 1).all())
    # expiration scan over a timers table of the same bucket count (one untimed scan first: the
    # table's pages are touched once before the timed scans)
    tt = FlowTable(table.n_buckets, timers=True, seed=seed, device=dev)
    tt.expire(100, stream)
    reps = 5
    e[0].record(stream)
    for r in range(reps):
        tt.expire(101 + r, stream)
    e[1].record(stream)
    e[1].synchronize()
    secs = e[0].elapsed_time(e[1]) / 1e3 / reps
    out["expire_scan_GBs"] = round(table.n_buckets * 64 / secs / 1e9, 1)
    del tt
    return out


def cpu_baseline(args, fill, q, nb, seed):
    """The CPU oracle (plain single-threaded C) on the same table and a bounded
    sample of the same lookup batch."""
    import oracle
    o = oracle.Table(nb, 8, False, seed)
    t0 = time.time()
    o.insert(fill.keys, fill.values)
    build_s = time.time() - t0
    sample = q.keys[: 1 << 21]
    done, t0 = 0, time.time()
    while time.time() - t0 < args.cpu_seconds:
        o.lookup(sample)
        done += sample.shape[0]
    secs = time.time() - t0
    o.close()
    return {"value": round(done / secs / 1e9, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} lookups ({sample.shape[0]}-key slices of the timed batch, neg {args.neg_rate}) "
                      f"on the oracle table of the same fill ({fill.keys.shape[0]} keys, built in {build_s:.0f} s)"}


def _share_nothing_worker(job):
    """One host core's share-nothing oracle table (spawned process, CPU only):
    build it, then time its lookups for `secs` seconds."""
    seed, log2_nb, lf, neg, secs = job
    import oracle
    from paper_1712_09624_gb300 import workload as W
    nb = 1 << log2_nb
    fill = W.fill(seed, int(lf * nb * 8))
    o = oracle.Table(nb, 8, False, seed)
    o.insert(fill.keys, fill.values)
    keys = W.lookup_batch(seed, 1 << 20, fill, neg).keys
    o.lookup(keys[: 1 << 16])
    done, t0 = 0, time.time()
    while time.time() - t0 < secs:
        o.lookup(keys)
        done += keys.shape[0]
    el = time.time() - t0
    o.close()
    return done, el


def cpu_baseline_share_nothing(args, log2_nb: int = 22, lf: float = 0.8, neg: float = 0.2, secs: float = 4.0):
    """The paper's multi-core setting (Sec. 5.3): one private oracle table per
    host core (2^22 buckets x 8 = 33.5M slots, LF 0.8, 20% negative lookups),
    all cores at once, each in its own spawned process; aggregate lookups/s."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    jobs = [(args.seed * 1000 + c, log2_nb, lf, neg, secs) for c in range(cores)]
    t0 = time.time()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_share_nothing_worker, jobs)
    value = sum(d / e for d, e in res)
    return {"value": round(value / 1e9, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one oracle table per core ({8 << log2_nb} slots, LF {lf}), 1M-key batches with {neg:.0%} "
                      f"negatives looked up for {secs:.0f} s per core; {time.time() - t0:.0f} s in all"}


# ------------------------------------------------------- reference arm

def run_reference(args):
    import oracle
    from paper_1712_09624_gb300 import workload as W
    nb = 1 << args.log2_buckets
    n_fill = int(args.load_factor * nb * 8)
    fill = W.fill(args.seed, n_fill)
    o = oracle.Table(nb, 8, False, args.seed)
    o.insert(fill.keys, fill.values)
    n = 1 << args.log2_batch
    q = W.lookup_batch(args.seed, n, fill, args.neg_rate)
    per_step = min(n, 1 << 20)  # bounded sample per step
    sample = q.keys[:per_step]
    for _ in range(args.warmup):
        o.lookup(sample)
    t0 = time.time()
    for _ in range(args.steps):
        v, f = o.lookup(sample)
    secs = time.time() - t0
    value = per_step * args.steps / secs / 1e9
    desc = f"{per_step} lookups per step from the {n}-key batch (neg {args.neg_rate}) on the oracle table " \
           f"({n_fill} keys, 2^{args.log2_buckets} buckets)"
    return {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": scale_config(args, n_fill),
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ------------------------------------------------------- batched form

def run_batched(args):
    """Batched form: args.tables tables with capacities log-uniform in [1K, 4M]
    slots at LF 0.85, each with a lookup batch log-uniform in [32, 64K] keys and
    30% negatives, served by one graph-captured persistent launch (autotuned)
    and, for comparison, by one plain ckpp_bulk_lookup launch per table (eager,
    and captured in one CUDA graph). All keys are drawn on the device by the
    workload generator; every output is checked against the workload's map."""
    import torch

    from paper_1712_09624_gb300 import _ckpp as K
    from paper_1712_09624_gb300 import workload_gpu as WG
    from paper_1712_09624_gb300.batched import BatchedLookup, autotune
    from paper_1712_09624_gb300.table import FlowTable

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(args.seed)
    nt = args.tables
    caps = np.exp(rng.uniform(np.log(1024), np.log(4 << 20), nt))
    nbs = np.maximum(2, np.round(caps / 8)).astype(np.int64)
    sizes = np.round(np.exp(rng.uniform(np.log(32), np.log(65536), nt))).astype(np.int64)
    fills = (0.85 * nbs * 8).astype(np.int64)
    t_build = time.time()
    ws = torch.empty(K.ckpp_workspace_bytes(int(fills.max())), dtype=torch.uint8, device=dev)
    tables, ok = [], torch.ones(1, dtype=torch.bool, device=dev)
    for i in range(nt):
        sd = args.seed * 100003 + i
        t = FlowTable(int(nbs[i]), seed=sd, device=dev)
        k, v = WG.fill_keys(sd, 0, int(fills[i]), dev)
        st = torch.empty(k.shape[0], dtype=torch.uint8, device=dev)
        K.ckpp_bulk_insert(t.handle, k, v, st, ws, 0, 0, stream)
        ok &= (st == K.ST_INSERTED).all()
        tables.append(t)
    jobs, expect = [], []
    for i in range(nt):
        sd = args.seed * 100003 + i
        kq, ef, ev = WG.lookup_batch(sd, int(sizes[i]), int(fills[i]), 0.3, 1, device=dev)
        jobs.append((i, kq, torch.empty(kq.shape[0], dtype=torch.int64, device=dev),
                     torch.empty(kq.shape[0], dtype=torch.uint8, device=dev)))
        expect.append((ef, ev))
    torch.cuda.synchronize()
    if not bool(ok.item()):
        raise RuntimeError("batched fill reported a status other than INSERTED")
    build_s = time.time() - t_build
    total = int(sizes.sum())
    batch = BatchedLookup(tables, max_jobs=nt, device=dev)
    batch.set_jobs(jobs)
    best, tune = autotune(batch, total)
    batch.capture(tuning=best)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3 / steps

    t_batched = timed(batch.replay, args.steps, args.warmup)
    good = all(bool(torch.equal(of, ef)) and bool(torch.equal(ov, ev))
               for (_, _, ov, of), (ef, ev) in zip(jobs, expect))
    lib = K.library()
    calls = [(t.handle, kq.data_ptr(), kq.shape[0], ov.data_ptr(), of.data_ptr())
             for t, (_, kq, ov, of) in zip(tables, jobs)]

    def plain():
        sh = stream.cuda_stream
        for h, kp, n, vp, fp in calls:
            lib.ckpp_bulk_lookup(h, kp, n, vp, fp, 0, 0, sh)

    for _, _, ov, of in jobs:
        ov.zero_()
        of.zero_()
    t_eager = timed(plain, max(3, args.steps // 20), 2)
    good_plain = all(bool(torch.equal(of, ef)) and bool(torch.equal(ov, ev))
                     for (_, _, ov, of), (ef, ev) in zip(jobs, expect))
    t_graph, graph_error = None, None
    try:
        g = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream(device=dev)
        cs.wait_stream(stream)
        with torch.cuda.stream(cs):
            with torch.cuda.graph(g, stream=cs, capture_error_mode="thread_local"):
                sh = cs.cuda_stream
                for h, kp, n, vp, fp in calls:
                    lib.ckpp_bulk_lookup(h, kp, n, vp, fp, 0, 0, sh)
        stream.wait_stream(cs)
        t_graph = timed(g.replay, max(5, args.steps // 5), 2)
    except Exception as e:  # report, do not hide, a capture failure
        graph_error = repr(e)[:200]
    slots = int(nbs.sum() * 8)
    return {
        "metric": "Glookups/s, batched form (many tables, one launch)", "value": round(total / t_batched / 1e9, 4),
        "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t_batched * 1e3, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"batched form: {nt} tables, capacities log-uniform [1K, 4M] slots, LF 0.85, "
                               "batches log-uniform [32, 64K] keys, 30% negatives",
                   "tables": nt, "total_slots": slots, "total_lookups_per_launch": total,
                   "table_bytes": int(sum(t.buf.numel() for t in tables)), "build_s": round(build_s, 1)},
        "tuning": {"threads_per_key": best[0], "group_depth": best[1], "blocks_per_sm": best[2],
                   "keys_per_warp": best[3],
                   "candidates_ms": {f"T{t}_G{gd}_B{b}": round(v * 1e3, 4) for (t, gd, b, kp), v in tune.items()}},
        "plain_per_table_eager": {"value": round(total / t_eager / 1e9, 4), "ms_per_step": round(t_eager * 1e3, 3)},
        "plain_per_table_graph": ({"value": round(total / t_graph / 1e9, 4), "ms_per_step": round(t_graph * 1e3, 3)}
                                  if t_graph else {"error": graph_error}),
        "speedup_vs_graph": round(t_graph / t_batched, 2) if t_graph else None,
        "speedup_vs_eager": round(t_eager / t_batched, 2),
        "results_match_map": good and good_plain, "gpu_launches": args.steps,
    }


# ------------------------------------------------------------- grid sweep

def run_sweep(args):
    """At-scale table (2^24 buckets x 8) filled step by step to LF 0.6, 0.7,
    0.8, 0.9, 0.95; at each LF, 16M-key lookups at negative rates 0, 0.25, 0.5,
    0.75, 1 with the three lookup strategies (Cuckoo++, optimistic,
    pessimistic). Reports Glookups/s, algorithmic bytes per lookup and the
    roofline fraction for every cell."""
    import torch

    from paper_1712_09624_gb300 import _ckpp as K
    from paper_1712_09624_gb300 import workload_gpu as WG
    from paper_1712_09624_gb300.table import FlowTable

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    nb = 1 << args.log2_buckets
    n = 1 << args.log2_batch
    peak, _ = measured_peaks()
    t = FlowTable(nb, seed=args.seed, device=dev)
    ws = torch.empty(K.ckpp_workspace_bytes(1 << 24), dtype=torch.uint8, device=dev)
    ov = torch.empty(n, dtype=torch.int64, device=dev)
    of = torch.empty(n, dtype=torch.uint8, device=dev)
    done, cells = 0, []
    names = {K.LOOKUP_BLOOM: "cuckoo++", K.LOOKUP_OPTIMISTIC: "optimistic", K.LOOKUP_PESSIMISTIC: "pessimistic"}
    for lf in (0.6, 0.7, 0.8, 0.9, 0.95):
        m = int(lf * nb * 8)
        while done < m:
            c = min(1 << 24, m - done)
            k, v = WG.fill_keys(args.seed, done, c, dev)
            st = torch.empty(c, dtype=torch.uint8, device=dev)
            K.ckpp_bulk_insert(t.handle, k, v, st, ws, 0, 0, stream)
            if not bool((st == K.ST_INSERTED).all()):
                raise RuntimeError(f"fill to LF {lf} reported a status other than INSERTED")
            done += c
        st = t.stats()
        for neg in (0.0, 0.25, 0.5, 0.75, 1.0):
            kq, ef, ev = WG.lookup_batch(args.seed, n, m, neg, int(lf * 100 + neg * 10), device=dev)
            for variant, name in names.items():
                cnt = torch.zeros(4, dtype=torch.int64, device=dev)
                K.ckpp_lookup_probe_counts(t.handle, kq, cnt, 0, variant, stream)
                reads = cnt.cpu().numpy()
                steps = max(5, args.steps // 10)
                for _ in range(3):
                    K.ckpp_bulk_lookup_variant(t.handle, kq, ov, of, 0, 0, variant, stream)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(steps):
                    K.ckpp_bulk_lookup_variant(t.handle, kq, ov, of, 0, 0, variant, stream)
                e1.record(stream)
                e1.synchronize()
                sec = e0.elapsed_time(e1) / 1e3 / steps
                exact = bool(torch.equal(of, ef)) and bool(torch.equal(ov, ev))
                b = alg_bytes_of(reads, n)
                cells.append({"lf": lf, "neg": neg, "strategy": name, "glookups": round(n / sec / 1e9, 3),
                              "alg_bytes_per_lookup": round(b / n, 2), "frac": round(b / sec / 1e9 / peak, 4),
                              "line_requests_per_lookup": round(lines_of(reads) / n, 4),
                              "secondary_reads_per_lookup": round(float(reads[1]) / n, 5), "exact": exact})
        cells[-1]["table"] = {"in_secondary": st["n_in_secondary"] / max(1, st["n_occupied"]),
                              "moved_zero": st["n_moved_zero"] / nb,
                              "fpr": st["bloom_pop_sq"] / (64.0 * 64.0 * nb)}
    headline = [c for c in cells if c["lf"] == 0.9 and c["neg"] == 0.5 and c["strategy"] == "cuckoo++"][0]
    return {"metric": METRIC + " (sweep)", "value": headline["glookups"], "unit": UNIT, "n_gpus": 1,
            "steps": max(5, args.steps // 10), "warmup": 3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "LF x negative-rate x strategy sweep, 2^24 buckets x 8, 16M-key batches",
                       "n_buckets": nb, "batch": n}, "cells": cells}


def run_served(args):
    """Served form: 64 ports of Poisson packet bursts (32..4096 keys, 2 G
    lookups/s offered, 10% inserts of new flows, 20% unknown flows) against
    256 tables of 500M slots in total, served by the continuous-batching loop
    and by one plain launch per burst; latency percentiles and throughput."""
    import torch

    from paper_1712_09624_gb300.serve import ServeConfig, Service
    torch.cuda.set_device(0)
    cfg = ServeConfig(duration_s=args.serve_seconds, seed=args.seed)
    if args.serve_flush_keys is not None:
        cfg.insert_flush_keys = args.serve_flush_keys
    if args.serve_flush_us is not None:
        cfg.insert_flush_s = args.serve_flush_us * 1e-6
    if args.serve_hold_us is not None:
        cfg.lookup_hold_s = args.serve_hold_us * 1e-6
    if args.serve_max_inflight is not None:
        cfg.max_inflight = args.serve_max_inflight
    if args.serve_one_stream:
        cfg.overlap = False
    out = {}
    for mode in args.serve_modes.split(","):
        svc = Service(cfg)
        r = svc.run(mode)
        r.update(svc.check())
        out[mode] = r
        del svc
        torch.cuda.empty_cache()
    b = out["batched"]
    return {"metric": "served Glookups/s and latency (continuous batching)", "value": b["achieved_glookups"],
            "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "served form: 64 ports, Poisson bursts of 32..4096 keys, 2 G lookups/s offered, "
                                   "256 tables / 500M slots, 10% inserts", "duration_s": cfg.duration_s,
                       "footprint_budget_bytes": cfg.footprint_bytes, "insert_flush_keys": cfg.insert_flush_keys,
                       "insert_flush_us": round(cfg.insert_flush_s * 1e6, 1),
                       "lookup_hold_us": round(cfg.lookup_hold_s * 1e6, 1), "raw_fraction": cfg.raw_fraction,
                       "max_inflight_turns": cfg.max_inflight, "overlap": cfg.overlap},
            "batched": b, "plain_per_burst": out.get("plain")}


def run_mixed(args):
    """Mixed mutation workload on one 200M-slot table with timers (25M buckets
    x 8). The warm fill reaches LF 0.9 with expiries spread over the next 1000
    time units. Then batches run, time +1 per batch, drawn 20:70:5:5 as:
    - insert 900K new flows (ttl 1000);
    - look up 4M keys, Zipf(0.99) over the live flows;
    - delete 250K live flows (uniform);
    - expire (full scan).
    A flow is named by its index in one global sequence of keys (the device
    generator, value = index), so the live window is known without host
    bookkeeping. Every batch's results are checked outside its timed region,
    against the sequential answer kept in a device map of deleted flows: every
    insert status is INSERTED (new flows); a lookup hits exactly the flows of
    the live window that no delete removed, with the flow's index as value;
    a delete batch reports DELETED for exactly its distinct flows that were
    still there. The warm fill's sub-batches expire in order (Sec. 4.2), and
    the window starts past the sub-batches whose expiry has passed."""
    import torch

    from paper_1712_09624_gb300 import _ckpp as K
    from paper_1712_09624_gb300 import workload_gpu as WG
    from paper_1712_09624_gb300.table import FlowTable

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(args.seed)
    nb = 25_000_000
    warm = int(0.9 * nb * 8)
    sub = 50  # warm sub-batches, expiries 20, 40, ..., 1000
    t = FlowTable(nb, timers=True, seed=args.seed, device=dev)
    ws = torch.empty(K.ckpp_workspace_bytes(1 << 22), dtype=torch.uint8, device=dev)
    per = (warm + sub - 1) // sub
    t_fill = time.time()
    for j in range(sub):
        lo = j * per
        n = min(per, warm - lo)
        for c in range(0, n, 1 << 22):
            m = min(1 << 22, n - c)
            k, v = WG.fill_keys(args.seed, lo + c, m, dev)
            st = torch.empty(m, dtype=torch.uint8, device=dev)
            K.ckpp_bulk_insert(t.handle, k, v, st, ws, 0, 20 * (j + 1), stream)
    torch.cuda.synchronize()
    fill_s = time.time() - t_fill
    # Zipf(0.99) ranks over [1, N] by the inverse of the continuous CDF approximation
    n_look, n_ins, n_del = 4_000_000, 900_000, 250_000
    s_exp = 0.99
    u = rng.random(n_look)
    big_n = float(warm)
    ranks = np.floor((1 + u * (big_n ** (1 - s_exp) - 1)) ** (1 / (1 - s_exp))).astype(np.int64) - 1
    ranks_d = torch.from_numpy(ranks).to(dev)
    mult = 0x9E3779B97F4A7C15 & ((1 << 63) - 1)
    ops = rng.choice(4, size=args.mixed_batches, p=[0.20, 0.70, 0.05, 0.05])
    next_flow = warm
    now = 0
    time_by = {0: 0.0, 1: 0.0, 2: 0.0, 3: 0.0}
    count_by = {0: 0, 1: 0, 2: 0, 3: 0}
    keys_by = {0: 0, 1: 0, 2: 0, 3: 0}
    hits = torch.zeros(1, dtype=torch.int64, device=dev)
    deleted = torch.zeros(1, dtype=torch.int64, device=dev)
    out_v = torch.empty(n_look, dtype=torch.int64, device=dev)
    out_f = torch.empty(n_look, dtype=torch.uint8, device=dev)
    st_ins = torch.empty(n_ins, dtype=torch.uint8, device=dev)
    st_del = torch.empty(n_del, dtype=torch.uint8, device=dev)
    n_expired = torch.zeros(1, dtype=torch.int64, device=dev)
    total_flows = warm + n_ins * int((ops == 0).sum())
    gone = torch.zeros(total_flows, dtype=torch.bool, device=dev)  # flows a delete removed
    bad = {"insert_status": torch.zeros(1, dtype=torch.int64, device=dev),
           "lookup": torch.zeros(1, dtype=torch.int64, device=dev),
           "delete_status": torch.zeros(1, dtype=torch.int64, device=dev)}
    hits_expected = torch.zeros(1, dtype=torch.int64, device=dev)
    for b, op in enumerate(ops):
        now += 1
        lo_live = min(warm, per * (now // 20))  # warm sub-batches whose expiry passed are dead
        window = next_flow - lo_live
        # inputs of this batch are prepared before its timed region
        if op == 0:
            k, v = WG.fill_keys(args.seed, next_flow, n_ins, dev)
            next_flow += n_ins
        elif op == 1:
            salt = int(rng.integers(0, 2**31))
            idx = lo_live + torch.remainder(ranks_d * mult + salt, window)
            k = WG.keys_at(args.seed, idx)
        elif op == 2:
            idx = torch.from_numpy(rng.integers(lo_live, next_flow, n_del)).to(dev)
            k = WG.keys_at(args.seed, idx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if op == 0:
            K.ckpp_bulk_insert(t.handle, k, v, st_ins, ws, now, 1000, stream)
        elif op == 1:
            K.ckpp_bulk_lookup(t.handle, k, out_v, out_f, now, 0, stream)
        elif op == 2:
            K.ckpp_bulk_delete(t.handle, k, st_del, ws, now, stream)
        else:
            K.ckpp_expire(t.handle, now, n_expired, stream)
        e1.record(stream)
        # checks, after the timed region on the same stream
        if op == 0:
            bad["insert_status"] += (st_ins != K.ST_INSERTED).sum()
        elif op == 1:
            want = ~gone[idx]
            hits += out_f.sum()
            hits_expected += want.sum()
            bad["lookup"] += ((out_f != want.to(torch.uint8)) | (want & (out_v != idx))).sum()
        elif op == 2:
            del_ok = st_del == K.ST_DELETED
            deleted += del_ok.sum()
            uniq = torch.unique(idx)
            # DELETED exactly once per distinct flow still there, never for a flow already gone
            bad["delete_status"] += (del_ok.sum() - (~gone[uniq]).sum()).abs() + (del_ok & gone[idx]).sum()
            gone[uniq] = True
        e1.synchronize()
        time_by[op] += e0.elapsed_time(e1) / 1e3
        count_by[op] += 1
        keys_by[op] += {0: n_ins, 1: n_look, 2: n_del, 3: nb}[op]
    torch.cuda.synchronize()
    st = t.stats(now)
    names = {0: "insert", 1: "lookup", 2: "delete", 3: "expire"}
    per_op = {names[o]: {"batches": count_by[o], "keys_or_buckets": keys_by[o],
                         "ms_per_batch": round(time_by[o] / max(1, count_by[o]) * 1e3, 4),
                         "per_s": round(keys_by[o] / max(time_by[o], 1e-12) / 1e6, 1)} for o in names}
    total_keys = keys_by[0] + keys_by[1] + keys_by[2]
    total_time = sum(time_by.values())
    return {"metric": "mixed insert/lookup/delete/expire: keys per second (GPU time)",
            "value": round(total_keys / total_time / 1e9, 4), "unit": "Gkeys/s", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "mixed mutation workload: 200M-slot table with timers, 20:70:5:5 "
                                   "insert/lookup/delete/expire batches, Zipf(0.99) lookups, ttl 1000",
                       "n_buckets": nb, "warm_entries": warm, "batches": int(args.mixed_batches),
                       "warm_fill_s": round(fill_s, 1)},
            "per_op": per_op, "lookup_hit_rate": round(float(hits.item()) / max(1, keys_by[1]), 4),
            "lookup_hit_rate_expected": round(float(hits_expected.item()) / max(1, keys_by[1]), 4),
            "mismatches": {k: int(v.item()) for k, v in bad.items()},
            "results_match": all(int(v.item()) == 0 for v in bad.values()) and t.sync_status() == 0,
            "deleted_live": int(deleted.item()), "expired": int(n_expired.item()),
            "table_after": {"live": st["n_live"], "occupied": st["n_occupied"],
                            "load_factor_live": round(st["n_live"] / (nb * 8), 4),
                            "in_secondary": round(st["n_in_secondary"] / max(1, st["n_occupied"]), 4)},
            "device_errors": t.sync_status()}


def run_insert_load(args):
    """Bulk insert rate as the table fills: a 2^24-bucket table (134M slots,
    no timers; --log2-buckets changes it) is filled to LF 0.85 untimed, then
    batches of 2^20 new keys are inserted until LF 0.99, each timed with CUDA
    events. Per batch: the load factor before it, the time, the statuses, and
    how many keys each displacement pass was left with (the workspace's
    diagnostic words)."""
    import torch

    from paper_1712_09624_gb300 import _ckpp as K
    from paper_1712_09624_gb300 import workload_gpu as WG
    from paper_1712_09624_gb300.table import FlowTable

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    nb = 1 << args.log2_buckets
    slots = nb * 8
    batch = 1 << 20
    t = FlowTable(nb, seed=args.seed, device=dev)
    ws = torch.empty(K.ckpp_workspace_bytes(1 << 22), dtype=torch.uint8, device=dev)
    done = 0
    warm = int(0.85 * slots)
    while done < warm:
        c = min(1 << 22, warm - done)
        k, v = WG.fill_keys(args.seed, done, c, dev)
        st = torch.empty(c, dtype=torch.uint8, device=dev)
        K.ckpp_bulk_insert(t.handle, k, v, st, ws, 0, 0, stream)
        done += c
    torch.cuda.synchronize()
    stored = warm
    rows = []
    st = torch.empty(batch, dtype=torch.uint8, device=dev)
    while stored < 0.99 * slots:
        k, v = WG.fill_keys(args.seed, done, batch, dev)
        done += batch
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        K.ckpp_bulk_insert(t.handle, k, v, st, ws, 0, 0, stream)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        diag = ws[:32].cpu().numpy().view(np.uint32)
        counts = np.bincount(st.cpu().numpy(), minlength=8)
        inserted = int(counts[K.ST_INSERTED])
        rows.append({"lf_before": round(stored / slots, 4), "ms": round(ms, 4),
                     "mkeys_per_s": round(batch / ms / 1e3, 1), "inserted": inserted,
                     "full": int(counts[K.ST_FULL]), "queued_by_phase1": int(diag[0]),
                     "left_after_one_move": int(diag[3]), "left_after_grid_search": int(diag[5]),
                     "left_after_second_pass": int(diag[6])})
        stored += inserted
    if t.sync_status() != 0:
        raise RuntimeError("a device wait gave up during the insert run")

    def rate(lo, hi):
        sel = [r for r in rows if lo <= r["lf_before"] < hi]
        return round(sum(batch for _ in sel) / max(1e-9, sum(r["ms"] for r in sel)) / 1e3, 1) if sel else None

    bands = {"0.85-0.90": rate(0.85, 0.90), "0.90-0.95": rate(0.90, 0.95), "0.95-0.99": rate(0.95, 0.99)}
    return {"metric": "bulk insert keys per second by load factor (GPU time)", "value": bands["0.85-0.90"],
            "unit": "Mkeys/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": f"bulk insert of 2^20-key batches of new keys into a 2^{args.log2_buckets}"
                                   "-bucket x 8 table from LF 0.85 to 0.99, no timers", "n_buckets": nb,
                                   "batch": batch},
            "bands_mkeys_per_s": bands, "rows": rows}


def main():
    args = parse()
    if args.record_traffic:
        record_traffic(args.record_traffic)
        return
    if args.workload != "scale" and args.impl == "ours":
        run = {"batched": run_batched, "sweep": run_sweep, "served": run_served, "mixed": run_mixed, "insert": run_insert_load}[args.workload]
        print(json.dumps(run(args)), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
