"""Batched form: lookups over many independent tables in one persistent launch.

``BatchedLookup`` describes a list of ``FlowTable``s to the library once
(``ckpp_batch_create``), keeps a device array of lookup jobs (one job = one
table's batch of keys and its output buffers), and launches the persistent
kernel over all jobs (``ckpp_batch_lookup``), eagerly or as a captured CUDA
graph that is replayed after the job array is rewritten.

``autotune`` times every kernel configuration (threads per key: 1, 2 or 4
lanes of a warp per key, i.e. 32, 16 or 8 keys per warp iteration; group
depth; persistent blocks per SM) on the current jobs with CUDA events and
keeps the fastest; results are cached per (device, job-count, key-count)
signature.
"""

from __future__ import annotations

import numpy as np
import torch

from . import _ckpp as K

JOB_DTYPE = np.dtype([("keys", "<u8"), ("out_vals", "<u8"), ("out_found", "<u8"), ("n", "<u4"), ("table", "<u4")])
assert JOB_DTYPE.itemsize == K.JOB_BYTES

THREADS_PER_KEY = [1, 2, 4]   # lanes of a warp per key; keys per warp iteration = 32 / threads_per_key
GROUP_DEPTHS = [1, 2]
BLOCKS_PER_SM = [1, 2, 3, 4]  # blocks of 512 threads

_tune_cache: dict[tuple, tuple[int, int, int, int]] = {}


class BatchedLookup:
    def __init__(self, tables, max_jobs: int | None = None, device=None, stream=None):
        self.tables = list(tables)
        self.device = torch.device(device) if device is not None else self.tables[0].device
        self.max_jobs = max_jobs or len(self.tables)
        if self.max_jobs > K.BATCH_MAX_JOBS:
            raise ValueError(f"at most {K.BATCH_MAX_JOBS} jobs per launch")
        self.desc = torch.empty(max(K.ckpp_batch_bytes(len(self.tables)), 256), dtype=torch.uint8, device=self.device)
        self.handle = K.ckpp_batch_create([t.handle for t in self.tables], self.desc, stream)
        self.jobs = torch.zeros(self.max_jobs * K.JOB_BYTES, dtype=torch.uint8, device=self.device)
        self.n_jobs = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.tuning: tuple[int, int, int, int] = (1, 1, 2, 32)
        self.graph = None
        self._keep = []

    def set_jobs(self, jobs, stream=None):
        """jobs: list of (table_index, keys [n,16] uint8, out_vals [n] int64, out_found [n] bool/uint8),
        all device tensors. Written into the device job array (stream-ordered)."""
        if len(jobs) > self.max_jobs:
            raise ValueError("more jobs than max_jobs")
        arr = np.zeros(self.max_jobs, JOB_DTYPE)
        for i, (ti, keys, ov, of) in enumerate(jobs):
            n = keys.shape[0]
            for name, t in (("keys", keys), ("out_vals", ov), ("out_found", of)):
                if not t.is_cuda or not t.is_contiguous():
                    raise ValueError(f"job {i}: {name} must be a contiguous CUDA tensor")
            if ov.shape[0] < n or of.shape[0] < n:
                raise ValueError(f"job {i}: outputs shorter than the keys")
            arr[i] = (keys.data_ptr(), ov.data_ptr(), of.data_ptr(), n, ti)
        host = torch.from_numpy(arr.view(np.uint8)).pin_memory()
        s = stream if stream is not None else torch.cuda.current_stream()
        with torch.cuda.stream(s):
            self.jobs.copy_(host, non_blocking=True)
            self.n_jobs.fill_(len(jobs))
        self._keep = [host, jobs]  # the pinned source and the tensors the jobs point at stay alive
        self.n_active = len(jobs)

    def launch(self, now: int = 0, tuning=None, stream=None):
        K.ckpp_batch_lookup(self.handle, self.jobs, self.max_jobs, self.n_jobs, now, tuning or self.tuning, stream)

    def capture(self, now: int = 0, tuning=None):
        """Capture one launch in a CUDA graph; replay() re-runs it on the current job array."""
        self.graph = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.launch(now, tuning, s)  # warm-up outside the capture
            s.synchronize()
            with torch.cuda.graph(self.graph, stream=s):
                self.launch(now, tuning, s)
        torch.cuda.current_stream().wait_stream(s)
        return self.graph

    def replay(self):
        self.graph.replay()

    def close(self):
        if getattr(self, "handle", None):
            K.ckpp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def time_launch(batch: BatchedLookup, tuning, reps: int = 5, now: int = 0) -> float:
    """Median seconds of one launch with `tuning` (CUDA events)."""
    stream = torch.cuda.current_stream()
    batch.launch(now, tuning, stream)
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.launch(now, tuning, stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    return float(np.median(times))


def autotune(batch: BatchedLookup, total_keys: int, now: int = 0,
             reps: int = 5) -> tuple[tuple[int, int, int, int], dict]:
    """Pick threads per key, group depth and blocks per SM by timing every
    configuration on the batch's current jobs. Returns (best, {config: seconds})
    with configs (threads_per_key, group_depth, blocks_per_sm, keys_per_warp)."""
    sig = (batch.device.index, batch.n_active, int(np.log2(max(total_keys, 1))))
    results = {}
    for tpk in THREADS_PER_KEY:
        for g in GROUP_DEPTHS:
            for bps in BLOCKS_PER_SM:
                cfg = (tpk, g, bps, 32 // tpk)
                results[cfg] = time_launch(batch, cfg, reps, now)
    best = min(results, key=results.get)
    _tune_cache[sig] = best
    batch.tuning = best
    return best, results
