"""FlowTable: a Cuckoo++ flow table in one torch-allocated device buffer.

A thin convenience layer over the C ABI (``_ckpp``): it owns the table's
device buffer and a reusable workspace, converts numpy inputs to device
tensors and allocates outputs. Every operation runs in libckpp's kernels.
"""

from __future__ import annotations

import numpy as np
import torch

from . import _ckpp as K


def as_device_keys(keys, device) -> torch.Tensor:
    if isinstance(keys, np.ndarray):
        keys = torch.from_numpy(np.ascontiguousarray(keys, dtype=np.uint8).reshape(-1, 16))
    if keys.dtype != torch.uint8 or keys.dim() != 2 or keys.shape[1] != 16:
        raise ValueError("keys must be uint8 [n, 16]")
    return keys.to(device, non_blocking=True).contiguous()


def as_device_values(values, device) -> torch.Tensor:
    if isinstance(values, np.ndarray):
        values = torch.from_numpy(np.ascontiguousarray(values).astype(np.uint64).view(np.int64))
    if values.dtype not in (torch.int64, torch.uint64):
        raise ValueError("values must be 64-bit integers")
    return values.to(device, non_blocking=True).contiguous()


class FlowTable:
    """A table of 8-slot buckets (capacity 8 * n_buckets) on one GPU."""

    def __init__(self, n_buckets: int, timers: bool = False, seed: int = 0, device=None, stream=None):
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.geo = K.geometry(n_buckets, timers, seed)
        nbytes = K.ckpp_required_bytes(self.geo)
        if nbytes == 0:
            raise ValueError(f"invalid geometry: n_buckets={n_buckets}")
        self.n_buckets, self.timers, self.seed = n_buckets, timers, seed
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.handle = K.ckpp_create(self.geo, self.buf, stream)
        self._ws = None

    @property
    def capacity(self) -> int:
        return self.n_buckets * K.SLOTS

    def workspace(self, n: int) -> torch.Tensor:
        need = K.ckpp_workspace_bytes(n)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        return self._ws

    def insert(self, keys, values, now: int = 0, ttl: int = 0, stream=None) -> torch.Tensor:
        k = as_device_keys(keys, self.device)
        v = as_device_values(values, self.device)
        status = torch.empty(k.shape[0], dtype=torch.uint8, device=self.device)
        K.ckpp_bulk_insert(self.handle, k, v, status, self.workspace(k.shape[0]), now, ttl, stream)
        return status

    def lookup(self, keys, now: int = 0, refresh_ttl: int = 0, stream=None):
        k = as_device_keys(keys, self.device)
        vals = torch.empty(k.shape[0], dtype=torch.int64, device=self.device)
        found = torch.empty(k.shape[0], dtype=torch.bool, device=self.device)
        K.ckpp_bulk_lookup(self.handle, k, vals, found, now, refresh_ttl, stream)
        return vals, found

    def delete(self, keys, now: int = 0, stream=None) -> torch.Tensor:
        k = as_device_keys(keys, self.device)
        status = torch.empty(k.shape[0], dtype=torch.uint8, device=self.device)
        K.ckpp_bulk_delete(self.handle, k, status, self.workspace(k.shape[0]), now, stream)
        return status

    def expire(self, now: int, stream=None) -> torch.Tensor:
        count = torch.zeros(1, dtype=torch.int64, device=self.device)
        K.ckpp_expire(self.handle, now, count, stream)
        return count

    def stats(self, now: int = 0, stream=None) -> dict:
        return K.ckpp_stats_get(self.handle, now, stream)

    def probe_counts(self, keys, now: int = 0, variant: int = K.LOOKUP_BLOOM, stream=None) -> torch.Tensor:
        """[primary bucket reads, secondary bucket reads, record reads,
        second-line reads] a lookup strategy makes on a batch."""
        k = as_device_keys(keys, self.device)
        counts = torch.zeros(4, dtype=torch.int64, device=self.device)
        K.ckpp_lookup_probe_counts(self.handle, k, counts, now, variant, stream)
        return counts

    def lookup_variant(self, keys, variant: int, now: int = 0, stream=None):
        """Lookup with an explicit strategy (Cuckoo++, optimistic, pessimistic)."""
        k = as_device_keys(keys, self.device)
        vals = torch.empty(k.shape[0], dtype=torch.int64, device=self.device)
        found = torch.empty(k.shape[0], dtype=torch.bool, device=self.device)
        K.ckpp_bulk_lookup_variant(self.handle, k, vals, found, now, 0, variant, stream)
        return vals, found

    def sync_status(self, stream=None) -> int:
        return K.ckpp_sync_status(self.handle, stream)

    def save(self, f, stream=None) -> None:
        """Checkpoint: the table's geometry and its whole device buffer, copied to
        host memory once the stream's queued work is done, written to f (a path
        or a file object) with torch.save."""
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        s.synchronize()
        torch.save({"n_buckets": self.n_buckets, "timers": self.timers, "seed": self.seed,
                    "bytes": self.buf.cpu()}, f)

    @classmethod
    def load(cls, f, device=None, now: int = 0, stream=None) -> "FlowTable":
        """Resume a table saved with save(): its bytes go to a new device buffer,
        opened with ckpp_attach (which checks the header). now: the time of the
        table's last expire scan (timers tables), from which the 64512-unit
        staleness window runs again."""
        d = torch.load(f)
        t = cls.__new__(cls)
        t.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        t.n_buckets, t.timers, t.seed = int(d["n_buckets"]), bool(d["timers"]), int(d["seed"])
        t.geo = K.geometry(t.n_buckets, t.timers, t.seed)
        t.buf = d["bytes"].to(t.device)
        t._ws = None
        t.handle = K.ckpp_attach(t.buf, now, stream)
        return t

    def close(self):
        if getattr(self, "handle", None):
            K.ckpp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
